"""Training stages around the Eq. 8 loss (Sec. 3.2.1, Table 1, Sec. 5).

* Parameter groups of each cell's weight blob: the six weight tensors of the
  C-cell (W1, W2, WL, P, WN, WD), and the literal cell's three branches
  split into their 3x3 taps (channels 0-7) and dilated taps (channels 8-11).
* Pre-process: the signs and scales of these groups fixed by Differential
  Evolution before training (DE/rand/1/bin, Storn & Price 1997), one signed
  scale per group.  Each candidate's loss is the Eq. 8 loss of one fixed
  batch of training windows, evaluated by libcloth (the loss alone, no
  backward sweep).  The random numbers come in as `draws`.
* Schedules of Table 1: step decay during training, cosine annealing for the
  fine-tuning stage.
* Branch-wise fine-tuning with the other branches frozen (Sec. 5): uint8
  masks for libcloth's masked Adam update.
"""
from __future__ import annotations

import math
import time

import numpy as np

C = 32
# the C-cell blob, in order (sizes from the layer shapes); bL is no scaling group
_CNN_LAYOUT = (("W1", C * 6 * 3 * 3), ("W2", C * C * 3 * 3), ("WL", 3 * C * 3 * 3), ("bL", 3), ("P", C * C),
               ("WN", 3 * C), ("WD", 3 * C))
_PCELL_NEAR, _PCELL_FAR = 8, 4   # channels per branch: 3x3 taps, dilated taps


def _cnn_spans():
    out, off = {}, 0
    for name, n in _CNN_LAYOUT:
        out[name] = (off, off + n)
        off += n
    return out


def _pcell_spans():
    out, off = {}, 0
    for br in ("L", "N", "D"):
        out[f"{br}_near"] = (off, off + _PCELL_NEAR)
        out[f"{br}_far"] = (off + _PCELL_NEAR, off + _PCELL_NEAR + _PCELL_FAR)
        off += _PCELL_NEAR + _PCELL_FAR
    out["b_L"] = (off, off + 3)
    return out


def scale_groups(cell: str) -> list[tuple[str, int, int]]:
    """The groups the pre-process scales: (name, first entry, end)."""
    if cell == "cnn":
        sp = _cnn_spans()
        return [(n, *sp[n]) for n in ("W1", "W2", "WL", "P", "WN", "WD")]
    if cell == "pcell":
        sp = _pcell_spans()
        return [(n, *sp[n]) for n in ("L_near", "L_far", "N_near", "N_far", "D_near", "D_far")]
    raise ValueError("cell must be 'cnn' or 'pcell'")


def mask_groups(cell: str) -> list[tuple[str, int, int]]:
    """Groups that fine-tuning can train or freeze: the scaling groups and
    the bias (bL of the C-cell, b_L of the literal cell)."""
    sp = _cnn_spans() if cell == "cnn" else _pcell_spans()
    bias = "bL" if cell == "cnn" else "b_L"
    return scale_groups(cell) + [(bias, *sp[bias])]


def scaled(w0, cell: str, x) -> np.ndarray:
    """float32 blob: group g of w0 times x[g] (product taken in float64)."""
    w = np.asarray(w0, dtype=np.float64).copy()
    groups = scale_groups(cell)
    if len(x) != len(groups):
        raise ValueError(f"{len(groups)} scales expected")
    for (_, a, b), s in zip(groups, x):
        w[a:b] *= float(s)
    return w.astype(np.float32)


def freeze_mask(cell: str, trainable, n: int) -> np.ndarray:
    """uint8 mask over n entries: 1 on the entries of the trainable groups."""
    spans = {name: (a, b) for name, a, b in mask_groups(cell)}
    mask = np.zeros(n, dtype=np.uint8)
    for name in trainable:
        if name not in spans:
            raise ValueError(f"unknown group {name!r} of the {cell} cell")
        a, b = spans[name]
        mask[a:b] = 1
    return mask


class StepLR:
    """lr0 * gamma ** (t // step_size) at iteration t (0-based)."""

    def __init__(self, lr0: float, step_size: int, gamma: float):
        if step_size < 1:
            raise ValueError("step_size >= 1")
        self.lr0, self.step_size, self.gamma = float(lr0), int(step_size), float(gamma)

    def __call__(self, t: int) -> float:
        return self.lr0 * self.gamma ** (int(t) // self.step_size)


class CosineLR:
    """Cosine annealing from lr0 at t = 0 to lr_min at t = T (held after T)."""

    def __init__(self, lr0: float, lr_min: float, T: int):
        if T < 1:
            raise ValueError("T >= 1")
        self.lr0, self.lr_min, self.T = float(lr0), float(lr_min), int(T)

    def __call__(self, t: int) -> float:
        t = min(int(t), self.T)
        return self.lr_min + 0.5 * (self.lr0 - self.lr_min) * (1.0 + math.cos(math.pi * t / self.T))


def differential_evolution(objective, lo, hi, draws, F: float = 0.5, CR: float = 0.9, first=None):
    """DE/rand/1/bin, vectorised over the population.  Generation g: mutants
    P[r1] + F (P[r2] - P[r3]) from the population at the generation's start,
    binomial crossover (component j from the mutant where cross < CR, and at
    jrand), trials clipped to [lo, hi], then each member replaced by its trial
    where the trial's objective is not larger.  Returns a dict: x, f (the
    best), history (best after each generation), population, fitness,
    initial_fitness (of the starting population), evals."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    P = lo + np.asarray(draws["init"], dtype=np.float64) * (hi - lo)
    NP, D = P.shape
    if first is not None:
        P[0] = np.asarray(first, dtype=np.float64)
    fit = np.array([float(objective(p)) for p in P])
    fit0 = fit.copy()
    evals = NP
    history = []
    rows = np.arange(NP)
    for g in range(np.asarray(draws["jrand"]).shape[0]):
        idx = np.asarray(draws["idx"][g])
        mutant = P[idx[:, 0]] + F * (P[idx[:, 1]] - P[idx[:, 2]])
        take = np.asarray(draws["cross"][g]) < CR
        take[rows, np.asarray(draws["jrand"][g])] = True
        trial = np.clip(np.where(take, mutant, P), lo, hi)
        ft = np.array([float(objective(u)) for u in trial])
        evals += NP
        keep = ft <= fit
        P = np.where(keep[:, None], trial, P)
        fit = np.where(keep, ft, fit)
        history.append(float(fit.min()))
    b = int(np.argmin(fit))
    return {"x": P[b].copy(), "f": float(fit[b]), "history": history, "population": P, "fitness": fit,
            "initial_fitness": fit0, "evals": evals}


class WindowLoss:
    """The Eq. 8 loss (alone) of one fixed batch of training windows, as a
    function of the group scales of a cell's blob: the pre-process objective.
    Non-finite losses (a scaling that makes the unroll blow up) count as
    +inf."""

    def __init__(self, cell: str, w0, specs, pins, x0, v0, targets, alpha: float = 0.5, g_norm: float = 9.81,
                 device="cuda", stride: int = 1):
        import torch

        from .cloth import ClothBatch
        from .net import FP32, Net

        self.cell, self.alpha, self.g_norm = cell, float(alpha), float(g_norm)
        self.w0 = np.asarray(w0, dtype=np.float32)
        self.S = int(targets.shape[0])
        self.targets = targets
        self.cb = ClothBatch(specs, pins, device=device)
        self.cb.set_state(x0, v0)
        if stride != 1:
            self.cb.set_net_stride(stride)
        self.net = Net(self.w0, FP32, device=device) if cell == "cnn" else None
        self.device = device
        self.calls = 0
        self._torch = torch

    def loss_of_blob(self, w) -> float:
        torch = self._torch
        wt = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).to(self.device)
        if self.cell == "cnn":
            self.net.set_weights(wt)
            loss, _ = self.cb.train_loss(self.net, self.S, self.targets, alpha=self.alpha, g_norm=self.g_norm,
                                         with_grad=False)
        else:
            loss, _ = self.cb.train_loss_pcell(wt, self.S, self.targets, alpha=self.alpha, g_norm=self.g_norm,
                                               with_grad=False)
        self.calls += 1
        v = float(loss.item())
        return v if math.isfinite(v) else math.inf

    def __call__(self, x) -> float:
        return self.loss_of_blob(scaled(self.w0, self.cell, x))

    def close(self) -> None:
        self.cb.close()
        if self.net is not None:
            self.net.close()


def de_preprocess(objective: WindowLoss, draws, bounds=(-4.0, 4.0), F: float = 0.5, CR: float = 0.9) -> dict:
    """Fix the group signs and scales by differential evolution (member 0
    starts at the unscaled blob, so the result is never worse than it).
    Returns the DE record plus the scaled blob (float32) and the wall time."""
    D = len(scale_groups(objective.cell))
    t0 = time.time()
    res = differential_evolution(objective, [bounds[0]] * D, [bounds[1]] * D, draws, F=F, CR=CR, first=np.ones(D))
    res["seconds"] = time.time() - t0
    res["blob"] = scaled(objective.w0, objective.cell, res["x"])
    res["groups"] = [g[0] for g in scale_groups(objective.cell)]
    return res
