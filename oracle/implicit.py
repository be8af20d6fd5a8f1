"""FP64 oracle of the implicit plain step (test infrastructure only).

Sec. 3.1 names implicit integration as the stable choice for large time
steps, and Sec. 5 lists larger-step and fully implicit integration as the
comparison for a larger-step cell.  This is the linearised backward Euler
step (one Newton step of v' = v + h M^-1 f(x + h v', v')), with the elastic
spring forces of Eq. 1 and the air drag of Eq. 4 implicit and the rest
(spring-axis damping of Eq. 2, pressure of Eq. 3, gravity) explicit:

  (m + h d) dv - h^2 K dv = h f(x, v) + h^2 K v,   v' = C(v + dv),
  x' = x + h v', then sphere contact (the update of Eq. 5),

where h is the step, K = df/dx of the springs, and for a spring (i, j) with
stiffness k, rest length L, d = x_j - x_i, l = |d|, n = d / l:
  K_ij = k [n n^T + max(0, 1 - L / l) (I - n n^T)] = -K_ii's share,
the transverse part clamped at zero under compression so that the matrix
stays symmetric positive definite.  Pinned nodes take dv = pin_v - v.  The
linear system is assembled as a sparse matrix and solved directly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# (row offset, column offset, spring type): structural, shear, bend
_SPRINGS = ((0, 1, 0), (1, 0, 0), (1, 1, 1), (1, -1, 1), (0, 2, 2), (2, 0, 2))


def springs(c: dict):
    """Every spring of the 13-point stencil once: arrays i, j, k, L."""
    rows, cols, h = int(c["rows"]), int(c["cols"]), float(c["h"])
    ks = (float(c["k_struct"]), float(c["k_shear"]), float(c["k_bend"]))
    I, J, K, L = [], [], [], []
    for dr, dc, t in _SPRINGS:
        for r in range(rows):
            for cc in range(cols):
                r2, c2 = r + dr, cc + dc
                if 0 <= r2 < rows and 0 <= c2 < cols:
                    I.append(r * cols + cc)
                    J.append(r2 * cols + c2)
                    K.append(ks[t])
                    L.append(h * float(np.hypot(dr, dc)))
    return np.array(I, dtype=np.int64), np.array(J, dtype=np.int64), np.array(K), np.array(L)


def stiffness(c: dict, x) -> sp.csr_matrix:
    """K = df/dx of the elastic springs (transverse part clamped at 0), as a
    sparse (3n, 3n) matrix."""
    rows, cols = int(c["rows"]), int(c["cols"])
    n = rows * cols
    X = np.asarray(x, dtype=np.float64).reshape(n, 3)
    I, J, kk, LL = springs(c)
    d = X[J] - X[I]
    ln = np.linalg.norm(d, axis=1)
    nn = d / ln[:, None]
    tr = np.maximum(0.0, 1.0 - LL / ln)
    blocks = kk[:, None, None] * (nn[:, :, None] * nn[:, None, :] +
                                  tr[:, None, None] * (np.eye(3)[None] - nn[:, :, None] * nn[:, None, :]))
    rr, cc_, vv = [], [], []
    for a in range(3):
        for b in range(3):
            blk = blocks[:, a, b]
            # f_i depends on x_j with +K_s, on x_i with -K_s; the same for f_j
            for (p, q, sgn) in ((I, J, 1.0), (J, I, 1.0), (I, I, -1.0), (J, J, -1.0)):
                rr.append(3 * p + a)
                cc_.append(3 * q + b)
                vv.append(sgn * blk)
    return sp.csr_matrix((np.concatenate(vv), (np.concatenate(rr), np.concatenate(cc_))), shape=(3 * n, 3 * n))


def implicit_step(c: dict, x, v, pins=(), steps: int = 1, stride: int = 1):
    """`steps` linearised backward Euler steps of h = stride dt (see the
    module docstring); returns new (x, v) of shape (rows, cols, 3)."""
    import oracle

    rows, cols = int(c["rows"]), int(c["cols"])
    n = rows * cols
    h = stride * float(c["dt"])
    m, drag = float(c["m"]), float(c.get("drag", 0.0))
    pin_v = np.asarray(c.get("pin_v", (0.0, 0.0, 0.0)), dtype=np.float64)
    pm = oracle.pin_mask(c, pins).astype(bool)
    free = np.repeat(~pm, 3)
    x = np.array(x, dtype=np.float64).reshape(rows, cols, 3)
    v = np.array(v, dtype=np.float64).reshape(rows, cols, 3)
    for _ in range(steps):
        f = oracle.total_force(c, x, v).reshape(-1)
        K = stiffness(c, x)
        vf = v.reshape(-1)
        A = sp.identity(3 * n, format="csr") * (m + h * drag) - (h * h) * K
        b = h * f + (h * h) * (K @ vf)
        dv = np.zeros(3 * n)
        dv[~free] = (np.broadcast_to(pin_v, (n, 3)).reshape(-1) - vf)[~free]
        rhs = b - A @ dv
        if free.any():
            Aff = A[free][:, free]
            dv[free] = spla.spsolve(Aff.tocsc(), rhs[free])
        # the update of Eq. 5 with the step h and the velocity change dv
        x, v = oracle.update(dict(c, dt=h), x, v, (dv / h).reshape(rows, cols, 3), pins)
    return x, v
