"""Training of the CNN cell on plain-simulator rollouts (Sec. 3.2.1, Eq. 8).

Host-side orchestration only: the trajectories are produced by libcloth's
plain step (recorded rollouts), the loss, its gradient through the 8-step
unroll and the Adam update run in libcloth's kernels.  The host samples the
windows (trajectory, start step) and gathers their states from the recorded
trajectories.
"""
from __future__ import annotations

import os

import numpy as np
import torch

from . import shard, stages
from . import workloads as wl
from .cloth import ClothBatch, pack
from .net import BF16, FP32, N_BLOB, N_PARAMS, Net, adam_step

# blob offsets of the linear branch's bias
_OFF_BL = 11808


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
        self.device = device

    def stats(self) -> dict:
        """Scales of the recorded data over the unpinned nodes of every step:
        root mean square of u = x - X and of v per coordinate, and mean and
        standard deviation per coordinate of the acceleration
        (v[t+1] - v[t]) / dt (which includes the small pressure term)."""
        d = self.device
        specs = self.cfg["specs"]
        n, h, dt = self.n, float(specs[0]["h"]), float(specs[0]["dt"])
        X = torch.zeros(n, n, 3, device=d, dtype=torch.float64)
        X[..., 0] = torch.arange(n, device=d, dtype=torch.float64)[None, :] * h
        X[..., 1] = torch.arange(n, device=d, dtype=torch.float64)[:, None] * h
        free = torch.ones(self.count, n * n, device=d, dtype=torch.float64)
        for b, pl in enumerate(self.cfg["pins"]):
            if len(pl):
                free[b, torch.as_tensor(list(pl), device=d)] = 0.0
        free = free.reshape(1, -1, 1)
        cnt = float(free.sum()) * self.steps
        su = torch.zeros(3, device=d, dtype=torch.float64)
        sv, sa, sa2 = torch.zeros_like(su), torch.zeros_like(su), torch.zeros_like(su)
        Xp = X.reshape(1, -1, 3).repeat(1, self.count, 1)
        for t0 in range(0, self.steps, 25):          # in slices: the recording is large
            t1 = min(self.steps, t0 + 25)
            x = self.x[t0:t1].double()
            v = self.v[t0:t1].double()
            a = (self.v[t0 + 1:t1 + 1].double() - v) / dt
            su += (((x - Xp) ** 2) * free).sum((0, 1))
            sv += ((v ** 2) * free).sum((0, 1))
            sa += (a * free).sum((0, 1))
            sa2 += ((a ** 2) * free).sum((0, 1))
        mean_a = sa / cnt
        return {"rms_u": (su / cnt).sqrt().tolist(), "rms_v": (sv / cnt).sqrt().tolist(),
                "mean_a": mean_a.tolist(), "std_a": (sa2 / cnt - mean_a ** 2).clamp_min(0).sqrt().tolist()}


def data_scaled_blob(stats: dict, seed: int = 2004) -> np.ndarray:
    """Initial C-cell weights scaled to the data (the input and output scales
    of the blob are free to be set from data statistics): in_scale = 1 / rms
    of u and v per coordinate, out_scale = the acceleration's standard
    deviation, b_L = its mean / out_scale, the other weights Kaiming (seed)."""
    ins = [1.0 / max(s, 1e-12) for s in stats["rms_u"]] + [1.0 / max(s, 1e-12) for s in stats["rms_v"]]
    outs = [max(s, 1e-6) for s in stats["std_a"]]
    blob = wl.kaiming_blob(seed, in_scale=ins, out_scale=outs)
    blob[_OFF_BL:_OFF_BL + 3] = np.asarray(stats["mean_a"]) / np.asarray(outs)
    return blob.astype(np.float32)


class StatePool:
    """Cloths stepped by the network being trained, whose states become
    training windows: the physics term of Eq. 8 compares the network's
    acceleration with the plain step's at any state, so states the network
    itself reaches (and drifts into) are labelled by the plain simulator as
    the recorded ones are (one plain step for the physics target, `unroll`
    plain steps for the data targets).  Each slot is one recorded cloth
    (its parameters and pins), restarted from a random recorded state of it
    when it has run `max_age` network steps or left the data's envelope
    (an in-plane displacement beyond `lim_u`, a speed beyond `lim_v`, or a
    non-finite value).  Not part of a checkpoint: a resumed trainer starts
    a new pool."""

    def __init__(self, data: Dataset, count: int, steps: int, max_age: int, lim_u: float, lim_v: float,
                 rng: np.random.Generator, device):
        self.data, self.steps, self.max_age, self.lim_u, self.lim_v = data, int(steps), int(max_age), lim_u, lim_v
        self.rng, self.device = rng, device
        self.count = min(int(count), data.count)
        self.ids = rng.choice(data.count, size=self.count, replace=False)
        self.specs = [data.cfg["specs"][i] for i in self.ids]
        self.pins = [data.cfg["pins"][i] for i in self.ids]
        nn = data.nodes
        self.idx = torch.from_numpy((self.ids[:, None] * nn + np.arange(nn)[None, :]).reshape(-1)).to(device)
        n, h = data.n, float(self.specs[0]["h"])
        X = torch.zeros(n, n, 3, device=device)
        X[..., 0] = torch.arange(n, device=device, dtype=torch.float32)[None, :] * h
        X[..., 1] = torch.arange(n, device=device, dtype=torch.float32)[:, None] * h
        self.X = X.reshape(1, nn, 3)
        self.cb = ClothBatch(self.specs, self.pins, device=device)
        self.x = data.x[0, self.idx].clone()
        self.v = data.v[0, self.idx].clone()
        self.age = np.zeros(self.count, dtype=np.int64)
        self.restarts = 0
        self.reset(np.arange(self.count))

    def reset(self, slots) -> None:
        slots = np.asarray(slots, dtype=np.int64)
        if slots.size == 0:
            return
        nn = self.data.nodes
        t = self.rng.integers(0, self.data.steps + 1, size=slots.size)
        rows = torch.from_numpy((slots[:, None] * nn + np.arange(nn)[None, :]).reshape(-1)).to(self.device)
        src = torch.from_numpy((self.ids[slots][:, None] * nn + np.arange(nn)[None, :]).reshape(-1)).to(self.device)
        tt = torch.from_numpy(np.repeat(t, nn)).to(self.device)
        self.x[rows] = self.data.x[tt, src]
        self.v[rows] = self.data.v[tt, src]
        self.age[slots] = 0
        self.restarts += int(slots.size)
        self.cb.set_state(self.x, self.v)

    def advance(self, net: Net) -> None:
        """`steps` network steps of every slot, then the restarts."""
        self.cb.step_net(net, self.steps)
        self.age += self.steps
        self.cb.get_state(self.x, self.v)
        nn = self.data.nodes
        u = (self.x.view(self.count, nn, 3) - self.X)[..., :2].abs().amax(dim=(1, 2))
        sp = self.v.view(self.count, nn, 3).abs().amax(dim=(1, 2))
        fin = torch.isfinite(self.x.view(self.count, -1)).all(dim=1) & torch.isfinite(self.v.view(self.count, -1)).all(dim=1)
        bad = (~fin) | (u > self.lim_u) | (sp > self.lim_v)
        bad = bad.cpu().numpy() | (self.age > self.max_age)
        self.reset(np.nonzero(bad)[0])

    def windows(self, k: int, unroll: int, stride: int):
        """k windows starting at distinct slots' current states, with the
        plain step's positions every `stride` steps as targets."""
        slots = self.rng.choice(self.count, size=k, replace=False)
        nn = self.data.nodes
        rows = torch.from_numpy((slots[:, None] * nn + np.arange(nn)[None, :]).reshape(-1)).to(self.device)
        specs = [self.specs[j] for j in slots]
        pins = [self.pins[j] for j in slots]
        x0, v0 = self.x[rows].contiguous(), self.v[rows].contiguous()
        sim = ClothBatch(specs, pins, device=self.device)
        sim.set_state(x0, v0)
        tg = torch.empty(unroll, k * nn, 3, device=self.device)
        sim.rollout(unroll * stride, record=tg, record_every=stride)
        sim.close()
        return specs, pins, x0, v0, tg

    def close(self) -> None:
        self.cb.close()


class Trainer:
    """Batches of `batch` windows, each an `unroll`-step stretch of one
    trajectory; Adam (Table 1) with lr 1e-3.  `cell` is "cnn" (the C-cell,
    FP32) or "pcell" (the literal cell: 39 trainable weights, alpha fixed).
    `lr_schedule` (a callable of the 0-based iteration, e.g. stages.StepLR or
    stages.CosineLR) replaces the constant lr; `trainable` (group names of
    stages.mask_groups) freezes every other group (branch-wise fine-tuning).
    `stride` k > 1 trains a larger-step cell: each network step spans k plain
    steps, so the window's targets are k plain steps apart.  Without `blob`
    the C-cell starts from data_scaled_blob of the dataset's statistics
    (init="data") or from Kaiming weights with input scales 1 / h and 1 s/m
    and output scale g (init="unit").  Under torch.distributed (`group`, or
    the default group once one is set up) every rank samples its own windows
    (seed + rank) and the gradients are averaged over the ranks before the
    identical Adam step.  With `pool` > 0 (C-cell only), from iteration
    `pool_warm` on a fraction `pool_frac` of every batch comes from a
    StatePool of that many cloths stepped `pool_steps` network steps per
    iteration (restarted after `pool_age` steps or outside 15 x the data's
    in-plane displacement and 20 x its speed)."""

    def __init__(self, data: Dataset, blob=None, batch: int = 64, unroll: int = 8, lr: float = 1e-3,
                 alpha: float = 0.5, seed: int = 7, device="cuda", cell: str = "cnn", lr_schedule=None,
                 trainable=None, stride: int = 1, init: str = "data", group=None, pool: int = 0,
                 pool_frac: float = 0.5, pool_steps: int = 4, pool_age: int = 800, pool_warm: int = 300):
        if cell not in ("cnn", "pcell"):
            raise ValueError("cell must be 'cnn' or 'pcell'")
        if stride < 1 or unroll * stride > data.steps:
            raise ValueError("need 1 <= stride and unroll * stride <= the recorded steps")
        self.stride = int(stride)
        self.data, self.batch, self.unroll, self.lr, self.alpha = data, batch, unroll, lr, alpha
        self.cell = cell
        import torch.distributed as dist
        self.group = group
        self.rank = dist.get_rank(group) if dist.is_available() and dist.is_initialized() else 0
        self.rng = np.random.default_rng(seed + self.rank)
        h = data.cfg["specs"][0]["h"]
        if init not in ("data", "unit"):
            raise ValueError("init must be 'data' or 'unit'")
        if blob is None:
            if cell == "pcell":
                blob = wl.pcell_blob(2006, h=h)
            elif init == "data":
                blob = data_scaled_blob(data.stats())
            else:
                blob = wl.kaiming_blob(2004, in_scale=(1.0 / h,) * 3 + (1.0,) * 3, out_scale=(9.81,) * 3)
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
        self.pool = None
        self.pool_cfg = None
        if pool > 0:
            if cell != "cnn":
                raise ValueError("the state pool serves the C-cell")
            if not 0.0 < pool_frac < 1.0:
                raise ValueError("pool_frac must lie in (0, 1)")
            st = data.stats()
            self.pool_cfg = {"count": int(pool), "frac": float(pool_frac), "steps": int(pool_steps),
                             "age": int(pool_age), "warm": int(pool_warm),
                             "lim_u": 15.0 * max(st["rms_u"][0], st["rms_u"][1]), "lim_v": 20.0 * max(st["rms_v"])}

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

    def sample_with_pool(self):
        """sample(), with the pool's share of the batch from the state pool
        once it is active."""
        pc = self.pool_cfg
        if pc is None or self.t < pc["warm"]:
            return self.sample()
        if self.pool is None:
            self.pool = StatePool(self.data, pc["count"], pc["steps"], pc["age"], pc["lim_u"], pc["lim_v"],
                                  self.rng, self.device)
        self.pool.advance(self.net)
        k = max(1, min(self.pool.count, int(round(pc["frac"] * self.batch))))
        full = self.batch
        self.batch = full - k
        try:
            specs, pins, x0, v0, tg = self.sample()
        finally:
            self.batch = full
        ps, pp, px, pv, pt = self.pool.windows(k, self.unroll, self.stride)
        return specs + ps, pins + pp, torch.cat([x0, px]), torch.cat([v0, pv]), torch.cat([tg, pt], dim=1)

    def step(self) -> float:
        if self.cell == "cnn":
            self.net.set_weights(self.w)
        specs, pins, x0, v0, tg = self.sample_with_pool()
        cb = ClothBatch(specs, pins, device=self.device)
        cb.set_state(x0, v0)
        if self.stride != 1:
            cb.set_net_stride(self.stride)
        if self.cell == "cnn":
            loss, g = cb.train_loss(self.net, self.unroll, tg, alpha=self.alpha)
        else:
            loss, g = cb.train_loss_pcell(self.w, self.unroll, tg, alpha=self.alpha)
        lr = self.lr_at(self.t)
        self.t += 1
        shard.average_gradient(g, self.batch, self.group)
        adam_step(self.w, g, self.m, self.v, self.t, lr=lr, n=self.n_params, mask=self.mask)
        cb.close()
        return float(loss.item())


# ------------------------------------------------------------- trained weights
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
TRAINED = os.path.join(DATA_DIR, "cnn_config4.npy")


def load_trained(path: str = TRAINED):
    """The committed C-cell weights of the training run (a float32 blob of
    13,036 values), or None when the file is absent."""
    if not os.path.exists(path):
        return None
    w = np.load(path).astype(np.float32)
    if w.shape != (N_BLOB,) or not np.all(np.isfinite(w)):
        raise ValueError(f"{path} is not a finite C-cell weight blob")
    return w


def gravity_only_blob(g=wl.G_DEFAULT) -> np.ndarray:
    """The zero network: every weight 0, b_L = g, unit scales, so a = g
    (free fall; the step still adds pressure, pins and contact)."""
    w = np.zeros(N_BLOB, dtype=np.float32)
    w[_OFF_BL:_OFF_BL + 3] = g
    w[N_PARAMS:] = 1.0
    return w


def evaluate(blobs: dict, cfg: dict, warm: int = 100, steps: int = 100, device="cuda", horizons=()) -> dict:
    """Accuracy of network rollouts against the plain step (Table 2's error):
    the cloths of `cfg` are first stepped `warm` plain steps, then each
    network of `blobs` ({name: (blob, precision)}) and the plain step run
    `steps` steps from that state.  Per network: the mean over nodes of
    |x_net - x_plain| / cloth width, and that error over the plain rollout's
    mean node displacement.  Also the displacement itself (relative to
    width).  `horizons` (step counts beyond `steps`) add the error relative
    to width at those horizons ("horizon_errors"; None once a network state
    is not finite)."""
    specs, pins = cfg["specs"], cfg["pins"]
    cb = ClothBatch(specs, pins, device=device)
    cb.set_state(pack(cfg["x"]).to(device), pack(cfg["v"]).to(device))
    cb.rollout(warm, graph_chunk=warm)
    x0, v0 = cb.get_state()
    marks = sorted({int(steps)} | {int(h) for h in horizons})
    plain = {}
    done = 0
    for h in marks:
        cb.rollout(h - done, graph_chunk=100)
        done = h
        plain[h] = cb.get_state()[0]
    widths = torch.tensor([(s["cols"] - 1) * s["h"] for s in specs], device=device, dtype=torch.float64)

    def per_cloth(a, b):
        return torch.stack([(p - q).double().norm(dim=1).mean() for p, q in zip(cb.split(a), cb.split(b))])

    disp = per_cloth(plain[steps], x0)
    out = {"warm_steps": warm, "steps": steps, "displacement_rel_width": float((disp / widths).mean())}
    for name, (blob, prec) in blobs.items():
        net = Net(blob, prec, device=device)
        cn = ClothBatch(specs, pins, device=device)
        cn.set_state(x0, v0)
        rec = {}
        done = 0
        for h in marks:
            cn.step_net(net, h - done)
            done = h
            xn, _ = cn.get_state()
            e = per_cloth(xn, plain[h])
            if h == steps:
                rec.update({"error_rel_width": float((e / widths).mean()),
                            "error_rel_displacement": float((e / disp).mean()),
                            "finite": bool(torch.isfinite(xn).all())})
            if h in horizons:
                ok = bool(torch.isfinite(xn).all())
                rec.setdefault("horizon_errors", {})[str(h)] = float((e / widths).mean()) if ok else None
        rec["status_word"] = cn.status()
        out[name] = rec
        cn.close()
        net.close()
    cb.close()
    return out


def main(argv=None) -> int:
    """Train the C-cell on the plain-simulator trajectories (512 cloths of
    64 x 64 x 200 steps, batch 64 windows, 8-step unroll, Adam from lr 1e-3
    with cosine annealing; from iteration 300 on half of each batch from a
    pool of 64 cloths stepped by the network, labelled by the plain step),
    checkpointing as it goes, then save the weights and a JSON record
    (losses, timing, held-out accuracy) beside them."""
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser(prog="python -m paper_2403_12820_gb300.train")
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-min", type=float, default=1e-5)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--unroll", type=int, default=8)
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--seed", type=int, default=1004)
    ap.add_argument("--out", default=TRAINED)
    ap.add_argument("--checkpoint", default=None, help="checkpoint file (default: <out>.ckpt.npz)")
    ap.add_argument("--checkpoint-every", type=int, default=500)
    ap.add_argument("--resume", action="store_true")
    ap.add_argument("--log-every", type=int, default=100)
    ap.add_argument("--eval-count", type=int, default=8, help="held-out 128 x 128 cloths for the accuracy check")
    ap.add_argument("--pool", type=int, default=64, help="cloths of the network-stepped state pool (0: none)")
    ap.add_argument("--pool-frac", type=float, default=0.5)
    ap.add_argument("--pool-steps", type=int, default=4)
    ap.add_argument("--pool-age", type=int, default=800)
    ap.add_argument("--pool-warm", type=int, default=300)
    a = ap.parse_args(argv)

    import torch.distributed as dist
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and not dist.is_initialized():
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    rank = dist.get_rank() if dist.is_initialized() else 0
    dev = torch.device("cuda", torch.cuda.current_device())
    ckpt = a.checkpoint or a.out + ".ckpt.npz"
    t0 = time.perf_counter()
    data = Dataset(count=a.count, n=a.n, steps=a.steps, seed=a.seed, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    stats = data.stats()
    tr = Trainer(data, batch=a.batch, unroll=a.unroll, lr=a.lr, device=dev,
                 lr_schedule=stages.CosineLR(a.lr, a.lr_min, a.iters), pool=a.pool, pool_frac=a.pool_frac,
                 pool_steps=a.pool_steps, pool_age=a.pool_age, pool_warm=a.pool_warm)
    if a.resume and os.path.exists(ckpt):
        tr.load(ckpt)
    log = []
    t1 = time.perf_counter()
    while tr.t < a.iters:
        loss = tr.step()
        if not np.isfinite(loss):
            raise RuntimeError(f"training diverged at iteration {tr.t}: loss {loss}")
        if tr.t % a.log_every == 0 or tr.t == 1 or tr.t == a.iters:
            log.append((tr.t, loss))
            if rank == 0:
                print(f"iter {tr.t} loss {loss:.5g} lr {tr.lr_at(tr.t - 1):.3g}", flush=True)
        if rank == 0 and a.checkpoint_every > 0 and tr.t % a.checkpoint_every == 0:
            tr.save(ckpt)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    if rank != 0:
        return 0
    w = tr.w.detach().cpu().numpy().astype(np.float32)
    g = data.cfg["specs"][0]["g"]
    ev = evaluate({"trained_fp32": (w, FP32), "trained_bf16": (w, BF16), "gravity_only": (gravity_only_blob(g), FP32)},
                  wl.cnn_batch(count=a.eval_count), device=dev, horizons=(200, 300, 500, 1000))
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.save(a.out, w)
    import sys
    rec = {"command": "python -m paper_2403_12820_gb300.train " + " ".join(sys.argv[1:] if argv is None else argv),
           "workload": f"{a.count} trajectories of {a.n} x {a.n} x {a.steps} plain steps (seed {a.seed}); batch "
                       f"{a.batch} windows, {a.unroll}-step unroll, Adam lr {a.lr} cosine to {a.lr_min}, "
                       f"{a.iters} iterations, alpha 0.5",
           "iterations": tr.t, "dataset_generation_s": gen_s, "train_s": train_s,
           "iters_per_s": a.iters / max(train_s, 1e-9), "loss_log": log, "data_stats": stats,
           "world_size": dist.get_world_size() if dist.is_initialized() else 1,
           "state_pool": dict(tr.pool_cfg, restarts=tr.pool.restarts if tr.pool is not None else 0)
           if tr.pool_cfg is not None else None,
           "held_out": dict(ev, workload=f"cnn_batch seed 1003, {a.eval_count} cloths of 128 x 128, "
                                         "after 100 plain steps")}
    with open(os.path.splitext(a.out)[0] + ".json", "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec["held_out"]), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
