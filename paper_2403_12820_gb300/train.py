"""Training of the CNN cell on plain-simulator rollouts (Sec. 3.2.1, Eq. 8).

Host-side orchestration only: the trajectories are produced by libcloth's
plain step (recorded rollouts), the loss, its gradient through the 8-step
unroll and the Adam update run in libcloth's kernels.  The host samples the
windows (trajectory, start step) and gathers their states from the recorded
trajectories.
"""
from __future__ import annotations

import numpy as np
import torch

from . import stages
from . import workloads as wl
from .cloth import ClothBatch, pack
from .net import FP32, N_BLOB, N_PARAMS, Net, adam_step


class Dataset:
    """`count` cloths of n x n stepped `steps` plain steps; positions and
    velocities of every step kept on the device: x[t], v[t] of shape
    (steps + 1, count * n * n, 3)."""

    def __init__(self, count: int = 512, n: int = 64, steps: int = 200, seed: int = 1004, device="cuda",
                 cfg: dict | None = None):
        self.cfg = cfg if cfg is not None else wl.train_cloths(seed=seed, count=count, n=n)
        self.count, self.n, self.steps = len(self.cfg["specs"]), int(self.cfg["specs"][0]["rows"]), int(steps)
        sim = ClothBatch(self.cfg["specs"], self.cfg["pins"], device=device)
        x0, v0 = pack(self.cfg["x"]).to(device), pack(self.cfg["v"]).to(device)
        N = sim.total_nodes
        self.x = torch.empty(steps + 1, N, 3, device=device)
        self.v = torch.empty(steps + 1, N, 3, device=device)
        self.x[0], self.v[0] = x0, v0
        sim.set_state(x0, v0)
        for t in range(1, steps + 1):
            sim.step(1)
            sim.get_state(self.x[t], self.v[t])
        sim.close()
        self.nodes = self.n * self.n


class Trainer:
    """Batches of `batch` windows, each an `unroll`-step stretch of one
    trajectory; Adam (Table 1) with lr 1e-3.  `cell` is "cnn" (the C-cell,
    FP32) or "pcell" (the literal cell: 39 trainable weights, alpha fixed).
    `lr_schedule` (a callable of the 0-based iteration, e.g. stages.StepLR or
    stages.CosineLR) replaces the constant lr; `trainable` (group names of
    stages.mask_groups) freezes every other group (branch-wise fine-tuning).
    `stride` k > 1 trains a larger-step cell: each network step spans k plain
    steps, so the window's targets are k plain steps apart."""

    def __init__(self, data: Dataset, blob=None, batch: int = 64, unroll: int = 8, lr: float = 1e-3,
                 alpha: float = 0.5, seed: int = 7, device="cuda", cell: str = "cnn", lr_schedule=None,
                 trainable=None, stride: int = 1):
        if cell not in ("cnn", "pcell"):
            raise ValueError("cell must be 'cnn' or 'pcell'")
        if stride < 1 or unroll * stride > data.steps:
            raise ValueError("need 1 <= stride and unroll * stride <= the recorded steps")
        self.stride = int(stride)
        self.data, self.batch, self.unroll, self.lr, self.alpha = data, batch, unroll, lr, alpha
        self.cell = cell
        self.rng = np.random.default_rng(seed)
        h = data.cfg["specs"][0]["h"]
        if blob is None:
            blob = (wl.kaiming_blob(2004, in_scale=(1.0 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3)
                    if cell == "cnn" else wl.pcell_blob(2006, h=h))
        self.w = torch.from_numpy(np.asarray(blob, dtype=np.float32)).to(device)
        self.n_params = N_PARAMS if cell == "cnn" else 39
        self.m = torch.zeros(self.n_params, device=device)
        self.v = torch.zeros(self.n_params, device=device)
        self.t = 0
        self.net = Net(blob, FP32, device=device) if cell == "cnn" else None
        self.device = device
        self.lr_schedule = lr_schedule
        self.mask = None
        self.set_trainable(trainable)

    def set_trainable(self, trainable=None) -> None:
        """Train only the named groups (None: every parameter)."""
        if trainable is None:
            self.mask = None
            return
        m = stages.freeze_mask(self.cell, trainable, self.n_params)
        self.mask = torch.from_numpy(m).to(self.device)

    def save(self, path: str) -> None:
        """Checkpoint: weights, Adam moments and step, the window sampler's
        random state and the cell kind, as one .npz file (the dataset and
        schedules are the caller's)."""
        import json
        np.savez(path, w=self.w.detach().cpu().numpy(), m=self.m.cpu().numpy(), v=self.v.cpu().numpy(),
                 t=np.int64(self.t), rng=np.array(json.dumps(self.rng.bit_generator.state)),
                 cell=np.array(self.cell))

    def load(self, path: str) -> None:
        """Resume from save(): the same cell on the same dataset continues
        bit for bit."""
        import json
        with np.load(path) as f:
            if str(f["cell"]) != self.cell:
                raise ValueError(f"checkpoint of the {f['cell']} cell, trainer of the {self.cell} cell")
            self.w.copy_(torch.from_numpy(f["w"]).to(self.device))
            self.m.copy_(torch.from_numpy(f["m"]).to(self.device))
            self.v.copy_(torch.from_numpy(f["v"]).to(self.device))
            self.t = int(f["t"])
            self.rng.bit_generator.state = json.loads(str(f["rng"]))

    def lr_at(self, t: int) -> float:
        return float(self.lr_schedule(t)) if self.lr_schedule is not None else self.lr

    def pre_process(self, draws, bounds=(-4.0, 4.0), F: float = 0.5, CR: float = 0.9) -> dict:
        """Differential-evolution pre-process (Sec. 3.2.1): fix the group signs
        and scales on one sampled batch of windows, apply them to the weights
        and restart Adam's moments.  Returns the DE record."""
        specs, pins, x0, v0, tg = self.sample()
        obj = stages.WindowLoss(self.cell, self.w.detach().cpu().numpy(), specs, pins, x0, v0, tg,
                                alpha=self.alpha, device=self.device, stride=self.stride)
        try:
            res = stages.de_preprocess(obj, draws, bounds=bounds, F=F, CR=CR)
        finally:
            obj.close()
        self.w.copy_(torch.from_numpy(res["blob"]).to(self.device))
        self.m.zero_()
        self.v.zero_()
        self.t = 0
        return res

    def sample(self):
        """Windows (trajectory, start) and a ClothBatch holding their cloths."""
        d = self.data
        traj = self.rng.choice(d.count, size=self.batch, replace=d.count < self.batch)
        start = self.rng.integers(0, d.steps - self.unroll * self.stride + 1, size=self.batch)
        specs = [d.cfg["specs"][i] for i in traj]
        pins = [d.cfg["pins"][i] for i in traj]
        nn = d.nodes
        idx = torch.from_numpy((traj[:, None] * nn + np.arange(nn)[None, :]).reshape(-1)).to(self.device)
        st = torch.from_numpy(np.repeat(start, nn)).to(self.device)
        x0 = d.x[st, idx].contiguous()
        v0 = d.v[st, idx].contiguous()
        tg = torch.stack([d.x[st + s * self.stride, idx] for s in range(1, self.unroll + 1)]).contiguous()
        return specs, pins, x0, v0, tg

    def step(self) -> float:
        specs, pins, x0, v0, tg = self.sample()
        cb = ClothBatch(specs, pins, device=self.device)
        cb.set_state(x0, v0)
        if self.stride != 1:
            cb.set_net_stride(self.stride)
        if self.cell == "cnn":
            self.net.set_weights(self.w)
            loss, g = cb.train_loss(self.net, self.unroll, tg, alpha=self.alpha)
        else:
            loss, g = cb.train_loss_pcell(self.w, self.unroll, tg, alpha=self.alpha)
        lr = self.lr_at(self.t)
        self.t += 1
        adam_step(self.w, g, self.m, self.v, self.t, lr=lr, n=self.n_params, mask=self.mask)
        cb.close()
        return float(loss.item())
