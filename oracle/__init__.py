"""FP64 CPU oracle for the cloth hot path (test infrastructure only).

This package is the slow, obviously correct statement of what the CUDA
library computes.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product path never does, and
it shares no code with the CUDA library.

The arithmetic lives in plain C files compiled on demand with gcc
(``cloth_oracle.c``: the mass-spring system of Sec. 3.1, Eq. 1-5;
``cnn_oracle.c``: the CNN cell of Sec. 3.2, Eq. 6-7 and its backward;
``pcell_oracle.c``: the cell of Eq. 6-7 read literally, with frozen
difference channels and ISRU).  This module marshals numpy arrays and
composes those primitives into the network step of Fig. 2 and the training
loss of Eq. 8, step by step.  ``stages.py`` (numpy) holds the training
stages around that loss (Sec. 3.2.1, Table 1): the differential-evolution
pre-process, the learning-rate schedules and the masked Adam update of
branch-wise fine-tuning; ``implicit.py`` (numpy, scipy.sparse) the
linearised backward Euler step, solved directly.

Array conventions: a cloth state is ``x, v`` of shape ``(rows, cols, 3)``
float64; node (r, c) rests at ``X = (c h, r h, 0)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["cloth_oracle.c", "cnn_oracle.c", "pcell_oracle.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_PARAMS = 13027   # trainable entries of the weight blob
N_BLOB = 13036     # + in_scale[6] + out_scale[3]
PCELL_BLOB = 40    # w_L[12], w_N[12], w_D[12], b_L[3], alpha
# channel c of the literal cell: (row offset, column offset) of its neighbour
PCELL_CHANNELS = ((0, 1), (0, -1), (1, 0), (-1, 0), (1, 1), (1, -1), (-1, 1), (-1, -1),
                  (0, 2), (0, -2), (2, 0), (-2, 0))


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, no FP contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= lib_m for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cloth(ctypes.Structure):
    _fields_ = [
        ("rows", ctypes.c_int32), ("cols", ctypes.c_int32),
        ("h", ctypes.c_double), ("m", ctypes.c_double),
        ("k_struct", ctypes.c_double), ("k_shear", ctypes.c_double), ("k_bend", ctypes.c_double),
        ("mu", ctypes.c_double), ("drag", ctypes.c_double), ("p", ctypes.c_double),
        ("g", ctypes.c_double * 3), ("dt", ctypes.c_double),
        ("sphere_on", ctypes.c_int32), ("sphere_c", ctypes.c_double * 3), ("sphere_r", ctypes.c_double),
        ("sphere_mu", ctypes.c_double), ("pin_v", ctypes.c_double * 3),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            dp = P(ctypes.c_double)
            cp = P(_Cloth)
            lib.oracle_neighbor_mask.argtypes = [ctypes.c_int32, ctypes.c_int32, P(ctypes.c_uint16)]
            lib.oracle_spring_counts.argtypes = [ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int64)]
            for name in ("oracle_internal_force", "oracle_total_force"):
                getattr(lib, name).argtypes = [cp, dp, dp, dp]
            lib.oracle_pressure_force.argtypes = [cp, dp, dp]
            lib.oracle_external_force.argtypes = [cp, dp, dp]
            lib.oracle_pressure_vjp.argtypes = [cp, dp, dp, dp]
            lib.oracle_step.argtypes = [cp, P(ctypes.c_uint8), dp, dp, ctypes.c_int32]
            lib.oracle_update.argtypes = [cp, P(ctypes.c_uint8), dp, dp, dp]
            lib.oracle_energy.argtypes = [cp, dp, dp]
            lib.oracle_energy.restype = ctypes.c_double
            lib.oracle_cnn_forward.argtypes = [dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, dp, dp]
            lib.oracle_cnn_backward.argtypes = [dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, dp, dp, dp, dp]
            lib.oracle_pcell_accel.argtypes = [ctypes.c_int32, ctypes.c_int32, dp, dp, dp, dp]
            lib.oracle_pcell_backward.argtypes = [ctypes.c_int32, ctypes.c_int32, dp, dp, dp, dp, dp, dp, dp]
            lib.oracle_cnn_param_count.restype = ctypes.c_int32
            lib.oracle_cnn_blob_count.restype = ctypes.c_int32
            assert lib.oracle_cnn_param_count() == N_PARAMS
            assert lib.oracle_cnn_blob_count() == N_BLOB
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cloth(c: dict) -> _Cloth:
    s = _Cloth()
    s.rows, s.cols = int(c["rows"]), int(c["cols"])
    s.h, s.m = float(c["h"]), float(c["m"])
    s.k_struct, s.k_shear, s.k_bend = float(c["k_struct"]), float(c["k_shear"]), float(c["k_bend"])
    s.mu, s.drag, s.p = float(c.get("mu", 0.0)), float(c.get("drag", 0.0)), float(c.get("p", 0.0))
    for a in range(3):
        s.g[a] = float(c["g"][a])
    s.dt = float(c.get("dt", 0.0))
    sph = c.get("sphere")
    s.sphere_mu = -1.0
    if sph is not None:
        s.sphere_on = 1
        for a in range(3):
            s.sphere_c[a] = float(sph["center"][a])
        s.sphere_r = float(sph["radius"])
        s.sphere_mu = float(sph.get("friction", -1.0))
    pv = c.get("pin_v", (0.0, 0.0, 0.0))
    for a in range(3):
        s.pin_v[a] = float(pv[a])
    return s


def _state(a, rows, cols) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    assert a.shape == (rows, cols, 3), a.shape
    return a


def rest_positions(c: dict) -> np.ndarray:
    """X of node (r, c) = (c h, r h, 0)."""
    rows, cols, h = int(c["rows"]), int(c["cols"]), float(c["h"])
    X = np.zeros((rows, cols, 3))
    X[..., 0] = np.arange(cols)[None, :] * h
    X[..., 1] = np.arange(rows)[:, None] * h
    return X


# ---------------------------------------------------------------- topology
def neighbor_mask(rows: int, cols: int) -> np.ndarray:
    """uint16 [rows][cols]; bit s set iff the s-th stencil neighbour exists."""
    out = np.zeros((rows, cols), dtype=np.uint16)
    _load().oracle_neighbor_mask(rows, cols, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)))
    return out


def spring_counts(rows: int, cols: int) -> tuple[int, int, int]:
    out = np.zeros(3, dtype=np.int64)
    _load().oracle_spring_counts(rows, cols, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return int(out[0]), int(out[1]), int(out[2])


# ---------------------------------------------------------------- forces
def _force(fn: str, c: dict, *arrs) -> np.ndarray:
    rows, cols = int(c["rows"]), int(c["cols"])
    ins = [_state(a, rows, cols) for a in arrs]
    f = np.zeros((rows, cols, 3))
    s = _cloth(c)
    getattr(_load(), fn)(ctypes.byref(s), *[_dptr(a) for a in ins], _dptr(f))
    return f


def internal_force(c: dict, x, v) -> np.ndarray:
    """Eq. 1 + Eq. 2."""
    return _force("oracle_internal_force", c, x, v)


def pressure_force(c: dict, x) -> np.ndarray:
    """Eq. 3 (1/4 reading)."""
    return _force("oracle_pressure_force", c, x)


def external_force(c: dict, v) -> np.ndarray:
    """Eq. 4."""
    return _force("oracle_external_force", c, v)


def total_force(c: dict, x, v) -> np.ndarray:
    """Eq. 1 + 2 + 3 + 4."""
    return _force("oracle_total_force", c, x, v)


def pressure_vjp(c: dict, x, gf) -> np.ndarray:
    """(d pressure_force / d x)^T gf."""
    return _force("oracle_pressure_vjp", c, x, gf)


def pin_mask(c: dict, pins) -> np.ndarray:
    m = np.zeros(int(c["rows"]) * int(c["cols"]), dtype=np.uint8)
    for p in pins:
        m[int(p)] = 1
    return m


def step(c: dict, x, v, pins=(), steps: int = 1):
    """`steps` plain steps (Eq. 5 with pins and sphere contact); returns new (x, v)."""
    rows, cols = int(c["rows"]), int(c["cols"])
    x = _state(x, rows, cols).copy()
    v = _state(v, rows, cols).copy()
    pm = pin_mask(c, pins)
    s = _cloth(c)
    _load().oracle_step(ctypes.byref(s), pm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                        _dptr(x), _dptr(v), int(steps))
    return x, v


def update(c: dict, x, v, acc, pins=()):
    """One Eq. 5 update for the acceleration `acc` (rows, cols, 3): pinned
    nodes take the pin velocity c["pin_v"] (default 0), then sphere contact
    (c["sphere"]["friction"]: < 0 or absent = the node stops, else Coulomb).
    Returns new (x, v)."""
    rows, cols = int(c["rows"]), int(c["cols"])
    x = _state(x, rows, cols).copy()
    v = _state(v, rows, cols).copy()
    acc = _state(acc, rows, cols)
    pm = pin_mask(c, pins)
    s = _cloth(c)
    _load().oracle_update(ctypes.byref(s), pm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dptr(acc),
                          _dptr(x), _dptr(v))
    return x, v


def mean_accel(c: dict, x0, v0, pins=(), k: int = 1) -> np.ndarray:
    """Physics target of a network step spanning k plain steps: the mean
    acceleration (v_k - v_0) / (k dt) of k oracle steps from (x0, v0), less
    the pressure acceleration at x0 (which the network step adds itself)."""
    _, vk = step(c, x0, v0, pins=pins, steps=k)
    return (vk - np.asarray(v0, dtype=np.float64)) / (k * float(c["dt"])) - pressure_force(c, x0) / float(c["m"])


def energy(c: dict, x, v) -> float:
    rows, cols = int(c["rows"]), int(c["cols"])
    x = _state(x, rows, cols)
    v = _state(v, rows, cols)
    s = _cloth(c)
    return float(_load().oracle_energy(ctypes.byref(s), _dptr(x), _dptr(v)))


# ---------------------------------------------------------------- CNN cell
def _blob(w) -> np.ndarray:
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    assert w.shape == (N_BLOB,), w.shape
    return w


def cnn_forward(w, z) -> np.ndarray:
    """a[N][3][H][W] from z[N][6][H][W] (Eq. 6-7)."""
    w = _blob(w)
    z = np.ascontiguousarray(np.asarray(z, dtype=np.float64))
    N, Cin, H, W = z.shape
    assert Cin == 6
    a = np.zeros((N, 3, H, W))
    _load().oracle_cnn_forward(_dptr(w), N, H, W, _dptr(z), _dptr(a))
    return a


def cnn_backward(w, z, ga):
    """(grad_w[13027], grad_z[N][6][H][W]) for cotangent ga[N][3][H][W]."""
    w = _blob(w)
    z = np.ascontiguousarray(np.asarray(z, dtype=np.float64))
    ga = np.ascontiguousarray(np.asarray(ga, dtype=np.float64))
    N, _, H, W = z.shape
    assert ga.shape == (N, 3, H, W)
    gw = np.zeros(N_PARAMS)
    gz = np.zeros_like(z)
    _load().oracle_cnn_backward(_dptr(w), N, H, W, _dptr(z), _dptr(ga), _dptr(gw), _dptr(gz))
    return gw, gz


def net_input(c: dict, x, v) -> np.ndarray:
    """z[1][6][rows][cols] = [u; v] with u = x - X."""
    u = np.asarray(x, dtype=np.float64) - rest_positions(c)
    z = np.concatenate([u, np.asarray(v, dtype=np.float64)], axis=2)   # rows, cols, 6
    return np.ascontiguousarray(z.transpose(2, 0, 1)[None])


def net_accel(w, c: dict, x, v) -> np.ndarray:
    """The cell's acceleration at every node, shape (rows, cols, 3)."""
    a = cnn_forward(w, net_input(c, x, v))[0]
    return np.ascontiguousarray(a.transpose(1, 2, 0))


def net_step(w, c: dict, x, v, pins=(), steps: int = 1):
    """Framework step of Fig. 2: network acceleration plus the hard-encoded
    pressure (Eq. 3) drive Eq. 5 with pins and sphere contact."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    for _ in range(steps):
        acc = net_accel(w, c, x, v) + pressure_force(c, x) / float(c["m"])
        x, v = update(c, x, v, acc, pins)
    return x, v


# ---------------------------------------------------------------- literal cell
def pcell_accel(w, c: dict, x, v) -> np.ndarray:
    """The cell of Eq. 6-7 read literally (Fig. 1): per coordinate, 12
    frozen difference channels phi_c = x_j - x_i, xi_c = v_j - v_i over the
    stencil neighbours that exist; a = sum_c [w_L phi + w_N sigma(phi) +
    w_D xi sigma(phi)] + b_L with the ISRU sigma.  Shape (rows, cols, 3)."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    assert w.shape == (PCELL_BLOB,), w.shape
    rows, cols = int(c["rows"]), int(c["cols"])
    x = _state(x, rows, cols)
    v = _state(v, rows, cols)
    a = np.zeros((rows, cols, 3))
    _load().oracle_pcell_accel(rows, cols, _dptr(w), _dptr(x), _dptr(v), _dptr(a))
    return a


def pcell_backward(w, c: dict, x, v, ga):
    """(grad_w[40] with grad_w[39] = 0 (alpha fixed), grad_x, grad_v) of
    sum(ga . pcell_accel(w, c, x, v)); shapes (rows, cols, 3)."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    assert w.shape == (PCELL_BLOB,), w.shape
    rows, cols = int(c["rows"]), int(c["cols"])
    x = _state(x, rows, cols)
    v = _state(v, rows, cols)
    ga = _state(ga, rows, cols)
    gw = np.zeros(PCELL_BLOB)
    gx = np.zeros((rows, cols, 3))
    gv = np.zeros((rows, cols, 3))
    _load().oracle_pcell_backward(rows, cols, _dptr(w), _dptr(x), _dptr(v), _dptr(ga), _dptr(gw), _dptr(gx),
                                  _dptr(gv))
    return gw, gx, gv


def pcell_step(w, c: dict, x, v, pins=(), steps: int = 1):
    """Framework step of Fig. 2 with the literal cell: its acceleration plus
    the hard-encoded pressure (Eq. 3) drive Eq. 5 with pins and sphere
    contact."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    for _ in range(steps):
        acc = pcell_accel(w, c, x, v) + pressure_force(c, x) / float(c["m"])
        x, v = update(c, x, v, acc, pins)
    return x, v


# ---------------------------------------------------------------- loss (Eq. 8)
def unroll_loss(w, c: dict, pins, x0, v0, x_targets, a_true, alpha: float, g_norm: float,
                h_norm: float, with_grad: bool = True, cell: str = "cnn"):
    """Training loss of Eq. 8 for one window, and its gradient.

    Physics term: alpha * mean over free nodes and 3 components of
    ((a_net(x0, v0) - a_true) / g_norm)^2.
    Data term: (1 - alpha) / S * sum_{s=1..S} mean over free nodes and
    components of ((x_hat_s - x_s) / h_norm)^2, where x_hat_s is the
    S-step unroll of `net_step` (no sphere) from (x0, v0).
    Returns (loss, grad_w) — grad by the hand-written adjoint of the
    unroll: Euler, pins, pressure and the cell's backward.  `cell` is "cnn"
    (the C-cell, grad_w[13027]) or "pcell" (the literal cell, grad_w[40]
    with the fixed alpha's entry 0).
    """
    assert cell in ("cnn", "pcell")
    accel = net_accel if cell == "cnn" else pcell_accel
    rows, cols = int(c["rows"]), int(c["cols"])
    dt, m = float(c["dt"]), float(c["m"])
    S = int(np.asarray(x_targets).shape[0])
    free = (1 - pin_mask(c, pins)).reshape(rows, cols, 1).astype(np.float64)
    pin_v = np.asarray(c.get("pin_v", (0.0, 0.0, 0.0)), dtype=np.float64)   # pinned nodes move with it
    cnt = 3.0 * free.sum()
    xs = [np.array(x0, dtype=np.float64)]
    vs = [np.array(v0, dtype=np.float64)]
    accs = []
    for t in range(S):
        a = accel(w, c, xs[t], vs[t])
        accs.append(a)
        vn = free * (vs[t] + dt * (a + pressure_force(c, xs[t]) / m)) + (1.0 - free) * pin_v
        vs.append(vn)
        xs.append(xs[t] + dt * vn)
    da = (accs[0] - np.asarray(a_true)) / g_norm
    loss_phys = alpha * float((free * da * da).sum()) / cnt
    loss_data = 0.0
    for s in range(1, S + 1):
        dx = (xs[s] - np.asarray(x_targets[s - 1])) / h_norm
        loss_data += float((free * dx * dx).sum()) / cnt
    loss = loss_phys + (1.0 - alpha) * loss_data / S
    if not with_grad:
        return loss, None

    gw = np.zeros(N_PARAMS if cell == "cnn" else PCELL_BLOB)
    gx = np.zeros((rows, cols, 3))
    gv = np.zeros((rows, cols, 3))
    for t in range(S, 0, -1):
        gx = gx + (1.0 - alpha) / S * 2.0 * free * (xs[t] - np.asarray(x_targets[t - 1])) / (h_norm ** 2 * cnt)
        gv = gv + dt * gx                        # x_t = x_{t-1} + dt v_t
        wv = free * gv                           # v_t = free * (v_{t-1} + dt (a + f_p / m))
        ga = dt * wv
        if t - 1 == 0:
            ga = ga + alpha * 2.0 * free * da / (g_norm * cnt)
        gx_prev = gx + pressure_vjp(c, xs[t - 1], dt * wv / m)
        gv_prev = wv
        if cell == "cnn":
            gwt, gz = cnn_backward(w, net_input(c, xs[t - 1], vs[t - 1]),
                                   np.ascontiguousarray(ga.transpose(2, 0, 1)[None]))
            gz = gz[0].transpose(1, 2, 0)        # rows, cols, 6
            gxc, gvc = gz[..., 0:3], gz[..., 3:6]   # u = x - X
        else:
            gwt, gxc, gvc = pcell_backward(w, c, xs[t - 1], vs[t - 1], ga)
        gw += gwt
        gx = gx_prev + gxc
        gv = gv_prev + gvc
    return loss, gw


def adam_step(theta, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


from .implicit import implicit_step, springs, stiffness  # noqa: E402,F401
from .stages import (CNN_GROUPS, PCELL_GROUPS, adam_step_masked, de_minimize, group_mask,  # noqa: E402,F401
                     lr_cosine, lr_step, scaled_blob)
