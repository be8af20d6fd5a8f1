"""Torch-facing wrapper of the cloth context (argument marshalling only).

Torch supplies device memory and the stream; every step runs in libcloth's
CUDA kernels.  A cloth is described by a dict with keys rows, cols, h, m,
k_struct, k_shear, k_bend, mu, drag, p, g (3 floats), and optionally
sphere = {center: (3 floats), radius, friction (< 0 or absent: the node
stops; >= 0: Coulomb mu)} and pin_v (3 floats, the velocity the pinned nodes
move with; default 0); the time step dt is shared by the batch.  States are float32 CUDA tensors of shape (total_nodes, 3), cloths
packed back to back, node (r, c) of a cloth at row r * cols + c.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import ClothGrid, ClothParams, ClothPins, ClothSphere, NetRolloutOpts, RolloutOpts


def _stream_handle(stream: torch.cuda.Stream | None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _require_cuda(t: torch.Tensor, name: str, dtype=torch.float32) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor")
    return t


class ClothBatch:
    """A batch of cloths of uneven sizes stepped by one launch per step."""

    def __init__(self, specs: list[dict], pins: list[list[int]] | None = None, dt: float | None = None,
                 device: str | torch.device = "cuda", stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("ClothBatch needs a CUDA device (libcloth has no CPU path)")
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.specs = list(specs)
        B = len(specs)
        self.B = B
        dt = float(dt if dt is not None else specs[0]["dt"])
        self.dt = dt
        grids = (ClothGrid * B)()
        params = (ClothParams * B)()
        spheres = (ClothSphere * B)()
        pin_arrs = []
        pin_structs = (ClothPins * B)()
        for b, s in enumerate(specs):
            grids[b] = ClothGrid(int(s["rows"]), int(s["cols"]), float(s["h"]), float(s["m"]))
            g = s.get("g", (0.0, 0.0, -9.81))
            params[b] = ClothParams(float(s["k_struct"]), float(s["k_shear"]), float(s["k_bend"]),
                                    float(s.get("mu", 0.0)), float(s.get("drag", 0.0)), float(s.get("p", 0.0)),
                                    (ctypes.c_float * 3)(*[float(a) for a in g]))
            sph = s.get("sphere")
            if sph is not None:
                spheres[b] = ClothSphere((ctypes.c_float * 3)(*[float(a) for a in sph["center"]]),
                                         float(sph["radius"]), 1, float(sph.get("friction", -1.0)))
            pl = list(pins[b]) if pins is not None else []
            arr = (ctypes.c_int32 * max(1, len(pl)))(*pl)
            pin_arrs.append(arr)
            pv = s.get("pin_v", (0.0, 0.0, 0.0))
            pin_structs[b] = ClothPins(len(pl), ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32)),
                                       (ctypes.c_float * 3)(*[float(a) for a in pv]))
        nbytes = ctypes.c_size_t()
        _lib.check("cloth_workspace_size", self.lib.cloth_workspace_size(B, grids, ctypes.byref(nbytes)))
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            self.stream = stream
            _lib.check("cloth_create", self.lib.cloth_create(
                ctypes.byref(h), B, grids, params, pin_structs, spheres, ctypes.c_float(dt),
                _ptr(self.workspace), nbytes, _stream_handle(stream)))
        self.handle = h
        nB, nn = ctypes.c_int32(), ctypes.c_int64()
        _lib.check("cloth_info", self.lib.cloth_info(h, ctypes.byref(nB), ctypes.byref(nn)))
        self.total_nodes = nn.value
        offs = [0]
        for s in specs:
            offs.append(offs[-1] + int(s["rows"]) * int(s["cols"]))
        self.node_offsets = offs

    # ----------------------------------------------------------- state
    def _s(self):
        return _stream_handle(self.stream)

    def set_state(self, x: torch.Tensor, v: torch.Tensor | None = None) -> None:
        _require_cuda(x, "x")
        if v is not None:
            _require_cuda(v, "v")
        if x.numel() != 3 * self.total_nodes or (v is not None and v.numel() != 3 * self.total_nodes):
            raise ValueError("state tensors must hold 3 * total_nodes floats")
        _lib.call("cloth_set_state", self.handle, _ptr(x), _ptr(v), self._s())

    def get_state(self, x: torch.Tensor | None = None, v: torch.Tensor | None = None):
        if x is None:
            x = torch.empty(self.total_nodes, 3, dtype=torch.float32, device=self.device)
        if v is None:
            v = torch.empty(self.total_nodes, 3, dtype=torch.float32, device=self.device)
        _lib.call("cloth_get_state", self.handle, _ptr(x), _ptr(v), self._s())
        return x, v

    def forces(self) -> torch.Tensor:
        f = torch.empty(self.total_nodes, 3, dtype=torch.float32, device=self.device)
        _lib.call("cloth_forces", self.handle, _ptr(f), self._s())
        return f

    def step(self, steps: int = 1) -> None:
        _lib.call("cloth_step_plain", self.handle, int(steps), self._s())

    def rollout(self, steps: int, graph_chunk: int = 0, record: torch.Tensor | None = None,
                record_every: int = 1) -> None:
        if record is not None:
            _require_cuda(record, "record")
            if record.numel() < (steps // record_every) * 3 * self.total_nodes:
                raise ValueError("record buffer too small")
        o = RolloutOpts(int(steps), int(graph_chunk), _ptr(record), int(record_every))
        _lib.call("cloth_rollout_plain", self.handle, ctypes.byref(o), self._s())

    def set_launch(self, seg_rows: int = 0, warps_per_sm: int = 0) -> None:
        _lib.call("cloth_set_launch", self.handle, int(seg_rows), int(warps_per_sm), self._s())

    def tune_launch(self, candidates: list[tuple[int, int]], warmup: int = 3, steps: int = 20) -> tuple[int, list[float]]:
        """Time each (seg_rows, warps_per_sm) candidate through cloth_tune_launch;
        the fastest is applied.  Returns (index of the fastest, us per step)."""
        n = len(candidates)
        seg = (ctypes.c_int32 * n)(*[int(c[0]) for c in candidates])
        wps = (ctypes.c_int32 * n)(*[int(c[1]) for c in candidates])
        us = (ctypes.c_float * n)()
        best = ctypes.c_int32()
        _lib.call("cloth_tune_launch", self.handle, n, seg, wps, int(warmup), int(steps), us, ctypes.byref(best),
                  self._s())
        return best.value, [float(v) for v in us]

    def step_implicit(self, steps: int, stride: int = 1, cg_iters: int = 20) -> None:
        """`steps` implicit (linearised backward Euler) plain steps of stride x dt."""
        n = ctypes.c_size_t()
        _lib.call("cloth_implicit_workspace_size", self.handle, ctypes.byref(n))
        ws = getattr(self, "_impl_ws", None)
        if ws is None or ws.numel() < n.value:
            ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            self._impl_ws = ws
        _lib.call("cloth_step_implicit", self.handle, int(steps), int(stride), int(cg_iters), _ptr(ws), ws.numel(),
                  self._s())

    def set_train_segment(self, k: int) -> None:
        """Keep every k-th unrolled state of the Eq. 8 loss (0: all) and
        recompute the rest in the backward sweep."""
        _lib.call("cloth_set_train_segment", self.handle, int(k))

    def set_net_stride(self, k: int) -> None:
        """One network step advances k plain time steps (dt_net = k dt)."""
        _lib.call("cloth_set_net_stride", self.handle, int(k), self._s())
        self.net_stride = int(k)

    def set_boundary(self, b: int, pin_v=(0.0, 0.0, 0.0), friction: float = -1.0) -> None:
        """Cloth b's pins move with pin_v (m/s) from the next step on, and its
        sphere contact takes `friction` (< 0: stick; >= 0: Coulomb mu)."""
        _lib.call("cloth_set_boundary", self.handle, int(b), (ctypes.c_float * 3)(*[float(a) for a in pin_v]),
                  ctypes.c_float(friction), self._s())

    def set_net_tile(self, precision: int, choice: int) -> None:
        """Tile shape of the network step for networks of `precision` (an
        index into tune.net_tile_choices(precision))."""
        _lib.call("cloth_set_net_tile", self.handle, int(precision), int(choice))

    def get_net_tile(self, precision: int) -> int:
        c = ctypes.c_int32()
        _lib.call("cloth_get_net_tile", self.handle, int(precision), ctypes.byref(c))
        return c.value

    def tune_net(self, net, warmup: int = 3, steps: int = 10) -> tuple[int, list[float]]:
        """Time the network step of `net` in every tile shape of its precision
        (cloth_tune_net; the state does not move) and apply the fastest.
        Returns (its choice index, us per step of each choice)."""
        ws = self.net_workspace(net.precision)
        us = (ctypes.c_float * 16)()
        best = ctypes.c_int32()
        _lib.call("cloth_tune_net", self.handle, net.handle, int(warmup), int(steps), us, ctypes.byref(best),
                  _ptr(ws), ws.numel(), self._s())
        from .tune import net_tile_choices
        n = len(net_tile_choices(net.precision))
        return best.value, [float(us[i]) for i in range(n)]

    def get_launch(self) -> tuple[int, int, int]:
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _lib.call("cloth_get_launch", self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return a.value, b.value, c.value

    def net_workspace(self, precision: int) -> torch.Tensor:
        n = ctypes.c_size_t()
        _lib.call("cloth_net_workspace_size", self.handle, int(precision), ctypes.byref(n))
        ws = getattr(self, "_net_ws", None)
        if ws is None or ws.numel() < n.value:
            ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            self._net_ws = ws
        return ws

    def step_net(self, net, steps: int = 1) -> None:
        """`steps` network steps (Fig. 2) with the given Net."""
        ws = self.net_workspace(net.precision)
        _lib.call("cloth_step_net", self.handle, net.handle, int(steps), _ptr(ws), ws.numel(), self._s())

    def rollout_net(self, net, steps: int, check_every: int = 0, residual_bound: float = 0.0,
                    graph_chunk: int = 0) -> None:
        """Network rollout (Fig. 2); every `check_every`-th step the plain step
        judges it and cloths whose largest node difference exceeds
        `residual_bound` (m) switch to the plain step."""
        n = ctypes.c_size_t()
        _lib.call("cloth_net_rollout_workspace_size", self.handle, int(net.precision), ctypes.byref(n))
        ws = getattr(self, "_roll_ws", None)
        if ws is None or ws.numel() < n.value:
            ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            self._roll_ws = ws
        o = NetRolloutOpts(int(steps), int(check_every), float(residual_bound), int(graph_chunk))
        _lib.call("cloth_rollout_net", self.handle, net.handle, ctypes.byref(o), _ptr(ws), ws.numel(), self._s())

    def _pcell_ws(self) -> torch.Tensor:
        n = ctypes.c_size_t()
        _lib.call("cloth_pcell_workspace_size", self.handle, ctypes.byref(n))
        ws = getattr(self, "_pcell_work", None)
        if ws is None or ws.numel() < n.value:
            ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            self._pcell_work = ws
        return ws

    @staticmethod
    def _pcell_w(w, device) -> torch.Tensor:
        w = torch.as_tensor(w, dtype=torch.float32).to(device).contiguous()
        if w.numel() != _lib.PCELL_BLOB:
            raise ValueError(f"literal-cell weights must hold {_lib.PCELL_BLOB} floats")
        return w

    def pcell_accel(self, w) -> torch.Tensor:
        """The literal cell's output (Eq. 6-7, Fig. 1) at the current state,
        packed (total_nodes, 3)."""
        w = self._pcell_w(w, self.device)
        ws = self._pcell_ws()
        a = torch.empty(self.total_nodes, 3, dtype=torch.float32, device=self.device)
        _lib.call("cloth_pcell_accel", self.handle, _ptr(w), _ptr(a), _ptr(ws), ws.numel(), self._s())
        return a

    def step_pcell(self, w, steps: int = 1) -> None:
        """`steps` network steps (Fig. 2) with the literal cell."""
        w = self._pcell_w(w, self.device)
        ws = self._pcell_ws()
        _lib.call("cloth_step_pcell", self.handle, _ptr(w), int(steps), _ptr(ws), ws.numel(), self._s())
        self._pcell_keep = w   # alive until the stream has used it

    def modes(self) -> tuple[torch.Tensor, torch.Tensor]:
        """(mode (B,) int32: 0 network, 1 plain; residual of the last check (B,) m)."""
        m = torch.empty(self.B, dtype=torch.int32, device=self.device)
        r = torch.empty(self.B, dtype=torch.float32, device=self.device)
        _lib.call("cloth_modes", self.handle, _ptr(m), _ptr(r), self._s())
        return m, r

    def reset_modes(self) -> None:
        _lib.call("cloth_reset_modes", self.handle, self._s())

    def train_loss(self, net, S: int, targets: torch.Tensor, alpha: float = 0.5, g_norm: float = 9.81,
                   grad_w: torch.Tensor | None = None, with_grad: bool = True):
        """Eq. 8 loss of the windows held by this batch (current state = window
        start) against `targets` (S, total_nodes, 3); adds its gradient to
        grad_w (created zero if None).  Returns (loss (1,), grad_w); with
        with_grad False only the loss (no backward sweep) and grad_w None."""
        _require_cuda(targets, "targets")
        if targets.numel() != S * 3 * self.total_nodes:
            raise ValueError("targets must hold S * total_nodes * 3 floats")
        n = ctypes.c_size_t()
        _lib.call("cloth_train_workspace_size", self.handle, int(S), ctypes.byref(n))
        ws = getattr(self, "_train_ws", None)
        if ws is None or ws.numel() < n.value:
            ws = torch.empty(n.value, dtype=torch.uint8, device=self.device)
            self._train_ws = ws
        if grad_w is None and with_grad:
            grad_w = torch.zeros(13027, dtype=torch.float32, device=self.device)
        if not with_grad:
            grad_w = None
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        _lib.call("cloth_train_loss", self.handle, net.handle, int(S), _ptr(targets), ctypes.c_float(alpha),
                  ctypes.c_float(g_norm), _ptr(loss), _ptr(grad_w), _ptr(ws), ws.numel(), self._s())
        return loss, grad_w

    def train_loss_pcell(self, w, S: int, targets: torch.Tensor, alpha: float = 0.5, g_norm: float = 9.81,
                         grad_w: torch.Tensor | None = None, with_grad: bool = True):
        """Eq. 8 with the literal cell (weights w, 40 floats): loss (1,) and
        grad_w (40,), the gradient added to the first 39 entries (None with
        with_grad False: the loss alone)."""
        _require_cuda(targets, "targets")
        if targets.numel() != S * 3 * self.total_nodes:
            raise ValueError("targets must hold S * total_nodes * 3 floats")
        w = self._pcell_w(w, self.device)
        n = ctypes.c_size_t()
        _lib.call("cloth_train_workspace_size", self.handle, int(S), ctypes.byref(n))
        ws = getattr(self, "_train_ws", None)
        if ws is None or ws.numel() < n.value:
            ws = torch.empty(n.value, dtype=torch.uint8, device=self.device)
            self._train_ws = ws
        if grad_w is None and with_grad:
            grad_w = torch.zeros(_lib.PCELL_BLOB, dtype=torch.float32, device=self.device)
        if not with_grad:
            grad_w = None
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        _lib.call("cloth_train_loss_pcell", self.handle, _ptr(w), int(S), _ptr(targets), ctypes.c_float(alpha),
                  ctypes.c_float(g_norm), _ptr(loss), _ptr(grad_w), _ptr(ws), ws.numel(), self._s())
        self._pcell_keep = w
        return loss, grad_w

    def topology(self, b: int) -> torch.Tensor:
        s = self.specs[b]
        m = torch.empty(int(s["rows"]) * int(s["cols"]), dtype=torch.int16, device=self.device)
        _lib.call("cloth_topology", self.handle, int(b), _ptr(m), self._s())
        return m

    def selftest_wait_timeout(self, polls: int = 1000) -> None:
        """Run the bounded-wait self-test (sets the timeout bit of the status word)."""
        _lib.call("cloth_selftest_wait_timeout", self.handle, int(polls), self._s())

    def status(self, clear: bool = False) -> int:
        st = ctypes.c_int32()
        _lib.call("cloth_status", self.handle, ctypes.byref(st), int(clear), self._s())
        return st.value

    def split(self, t: torch.Tensor) -> list[torch.Tensor]:
        """Per-cloth views (rows, cols, 3) of a packed (total_nodes, 3) tensor."""
        out = []
        for b, s in enumerate(self.specs):
            a, e = self.node_offsets[b], self.node_offsets[b + 1]
            out.append(t[a:e].view(int(s["rows"]), int(s["cols"]), 3))
        return out

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.lib.cloth_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack(arrs) -> torch.Tensor:
    """Concatenate per-cloth (rows, cols, 3) float32 arrays into (total_nodes, 3)."""
    import numpy as np
    return torch.from_numpy(np.concatenate([np.asarray(a, dtype=np.float32).reshape(-1, 3) for a in arrs]))
