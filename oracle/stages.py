"""FP64 oracle of the training stages around the Eq. 8 loss (test
infrastructure only): Sec. 3.2.1 and Table 1.

* Pre-process: the signs and scales of the branch parameter groups fixed by
  Differential Evolution before training (DE/rand/1/bin of Storn & Price,
  1997): a population of candidate group-scale vectors; for every member a
  mutant x_r1 + F (x_r2 - x_r3) from three other members, binomial crossover
  with the member (each component from the mutant with probability CR, one
  component always), and greedy selection of the trial where its loss is not
  larger.  The random numbers are inputs (`draws`), so a run is reproducible.
* Post-process: the learning-rate schedules of Table 1 (step decay during
  training, cosine annealing for the fine-tuning stage).
* Branch-wise fine-tuning with the other branches frozen (Sec. 5): an Adam
  update that leaves frozen entries (and their moments) untouched.

Group tables (entries of the weight blobs):
  C-cell blob: W1 [0, 1728), W2 [1728, 10944), WL [10944, 11808),
    P [11811, 12835), WN [12835, 12931), WD [12931, 13027)
    (bL [11808, 11811) and the in/out scales are in no group);
  literal cell blob: w_L near (3x3 taps, channels 0-7) [0, 8), w_L far
    (dilated taps, channels 8-11) [8, 12), then the same for w_N [12, 24) and
    w_D [24, 36) (b_L and alpha are in no group).
"""
from __future__ import annotations

import math

import numpy as np

CNN_GROUPS = (("W1", 0, 1728), ("W2", 1728, 10944), ("WL", 10944, 11808), ("P", 11811, 12835),
              ("WN", 12835, 12931), ("WD", 12931, 13027))
PCELL_GROUPS = (("L_near", 0, 8), ("L_far", 8, 12), ("N_near", 12, 20), ("N_far", 20, 24),
                ("D_near", 24, 32), ("D_far", 32, 36))


def groups(cell: str):
    assert cell in ("cnn", "pcell")
    return CNN_GROUPS if cell == "cnn" else PCELL_GROUPS


def scaled_blob(w, cell: str, x):
    """The blob with group g's entries multiplied by x[g] (all other entries
    as they are)."""
    out = np.array(w, dtype=np.float64)
    g = groups(cell)
    assert len(x) == len(g)
    for (name, a, b), s in zip(g, x):
        out[a:b] = out[a:b] * float(s)
    return out


def group_mask(n: int, cell: str, trainable) -> np.ndarray:
    """Boolean mask over n entries: True for the entries of the named groups."""
    mask = np.zeros(n, dtype=bool)
    names = set(trainable)
    for name, a, b in groups(cell):
        if name in names:
            mask[a:b] = True
            names.discard(name)
    assert not names, names
    return mask


def de_minimize(f, lo, hi, draws, F: float, CR: float, first=None):
    """DE/rand/1/bin over the box [lo, hi].

    draws: init (NP, D) uniforms: member i starts at lo + init_i (hi - lo)
      (member 0 at `first` when given); idx (G, NP, 3): r1, r2, r3 of member
      i in generation g; jrand (G, NP): the component always taken from the
      mutant; cross (G, NP, D) uniforms of the crossover.
    Within a generation every mutant is built from the population as it was
    at the generation's start; trials are clipped to the box.
    Returns (best x, best f, best f after each generation, population, f of
    the population, number of evaluations).
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    init = np.asarray(draws["init"], dtype=np.float64)
    NP, D = init.shape
    pop = lo + init * (hi - lo)
    if first is not None:
        pop[0] = np.asarray(first, dtype=np.float64)
    fit = np.array([float(f(pop[i])) for i in range(NP)])
    evals = NP
    history = []
    G = np.asarray(draws["jrand"]).shape[0]
    for g in range(G):
        old = pop.copy()
        new_pop = pop.copy()
        new_fit = fit.copy()
        for i in range(NP):
            r1, r2, r3 = (int(k) for k in draws["idx"][g][i])
            assert len({i, r1, r2, r3}) == 4
            mutant = old[r1] + F * (old[r2] - old[r3])
            trial = old[i].copy()
            for j in range(D):
                if draws["cross"][g][i][j] < CR or j == int(draws["jrand"][g][i]):
                    trial[j] = mutant[j]
            trial = np.minimum(np.maximum(trial, lo), hi)
            ft = float(f(trial))
            evals += 1
            if ft <= fit[i]:
                new_pop[i] = trial
                new_fit[i] = ft
        pop, fit = new_pop, new_fit
        history.append(float(fit.min()))
    b = int(np.argmin(fit))
    return pop[b].copy(), float(fit[b]), history, pop, fit, evals


def lr_step(lr0: float, step_size: int, gamma: float, t: int) -> float:
    """Step decay: lr0 gamma^floor(t / step_size) at (0-based) iteration t."""
    return lr0 * gamma ** (t // step_size)


def lr_cosine(lr0: float, lr_min: float, T: int, t: int) -> float:
    """Cosine annealing from lr0 (t = 0) to lr_min (t = T)."""
    return lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * t / T))


def adam_step_masked(theta, grad, m, v, t: int, lr: float, mask, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015, Algorithm 1) on the entries where mask is True;
    the others keep theta, m and v.  Returns (theta, m, v)."""
    theta, m, v = (np.array(a, dtype=np.float64) for a in (theta, m, v))
    k = np.asarray(mask, dtype=bool)
    g = np.asarray(grad, dtype=np.float64)
    m[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
    v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k]
    mh = m[k] / (1.0 - beta1 ** t)
    vh = v[k] / (1.0 - beta2 ** t)
    theta[k] = theta[k] - lr * mh / (np.sqrt(vh) + eps)
    return theta, m, v
