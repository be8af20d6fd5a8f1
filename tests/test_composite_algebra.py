"""The algebra the network-step kernels rely on, restated in FP64 NumPy and
checked against the layered oracle (Eq. 6-7).

The trunk W2 (*) (W1 (*) z) is linear and bias-free and phi enters Eq. 7
only through P and WL, so per node t = P phi, q_tap = WL_tap phi and xi
follow from one 5x5 composite kernel C_c = sum_{a+b=c} W2_a W1_b applied to
the zero-padded input.  The layers' own zero padding makes that differ on
the outermost ring of nodes; the kernels remove, per edge the node lies on,
the terms through the layer-1 positions outside the cloth (a 5-tap kernel
along the edge) and add back, where two edges meet, the term both removed.
These tests check that this restatement equals the oracle's layered cell to
rounding on grids from 1 x 1 up, and that each correction is needed.  They
use no part of the CUDA path.
"""
import numpy as np
import pytest

import oracle
from paper_2403_12820_gb300 import workloads as wl

kC = 32
# blob layout (include/cloth.h, CLOTH_NET_BLOB): W1[32][6][3][3], W2[32][32][3][3],
# WL[3][32][3][3], bL[3], P[32][32], WN[3][32], WD[3][32], in_scale[6], out_scale[3]
oW1 = 0
oW2 = oW1 + kC * 6 * 9
oWL = oW2 + kC * kC * 9
oBL = oWL + 3 * kC * 9
oP = oBL + 3
oWN = oP + kC * kC
oWD = oWN + 3 * kC
oIns = oWD + 3 * kC
oOuts = oIns + 6


def _terms(w):
    """Composite kernel C[cy][cx] and the edge (KE) and corner (KC) terms as
    [96 outputs][6 inputs] maps: outputs 0-31 t = P phi, 32-58 q (tap-major,
    then output coordinate), 64-95 xi; t and q read u, xi reads v."""
    W1 = w[oW1:oW2].reshape(kC, 6, 3, 3)
    W2 = w[oW2:oWL].reshape(kC, kC, 3, 3)
    WL = w[oWL:oBL].reshape(3, kC, 3, 3)
    P = w[oP:oWN].reshape(kC, kC)
    G = np.zeros((59, kC))
    G[:32] = P
    for m in range(27):
        tl, co = divmod(m, 3)
        G[32 + m] = WL[co, :, tl // 3, tl % 3]
    D = np.einsum('kjab,jicd->abcdki', W2, W1)   # W2_a W1_b: [ay][ax][by][bx][k][i]

    def gd(a, b):
        out = np.zeros((96, 6))
        Dab = D[a[0], a[1], b[0], b[1]]
        out[:59, :3] = G @ Dab[:, :3]
        out[64:, 3:] = Dab[:, 3:]
        return out

    C = np.zeros((5, 5, 96, 6))
    for ay in range(3):
        for ax in range(3):
            for by in range(3):
                for bx in range(3):
                    C[ay + by, ax + bx] += gd((ay, ax), (by, bx))
    # edges x = 0, x = W-1, y = 0, y = H-1: the outside layer-1 line a and the
    # only tap b that reaches back into the cloth, summed along the edge
    KE = np.zeros((4, 5, 96, 6))
    for ed in range(4):
        for s in range(5):
            for k in range(3):
                m = s - k
                if 0 <= m <= 2:
                    a, b = [((k, 0), (m, 2)), ((k, 2), (m, 0)), ((0, k), (2, m)), ((2, k), (0, m))][ed]
                    KE[ed, s] -= gd(a, b)
    KC = np.zeros((2, 2, 96, 6))   # [ay / 2][ax / 2]
    for yb in range(2):
        for xb in range(2):
            ay, ax = 2 * yb, 2 * xb
            KC[yb, xb] = gd((ay, ax), (2 - ay, 2 - ax))
    return C, KE, KC


def composite_cell(w, z, edges=True, corners=True):
    """a[N][3][H][W] by the composite restatement."""
    C, KE, KC = _terms(w)
    N, _, H, W = z.shape
    ins, outs, bL = w[oIns:oIns + 6], w[oOuts:oOuts + 3], w[oBL:oBL + 3]
    WN = w[oWN:oWD].reshape(3, kC)
    WD = w[oWD:oIns].reshape(3, kC)
    a = np.zeros((N, 3, H, W))
    for n in range(N):
        zp = np.zeros((6, H + 4, W + 4))
        zp[:, 2:H + 2, 2:W + 2] = z[n] * ins[:, None, None]
        Y = np.zeros((H, W, 96))
        for cy in range(5):
            for cx in range(5):
                Y += np.einsum('ni,iyx->yxn', C[cy, cx], zp[:, cy:cy + H, cx:cx + W])
        for y in range(H):
            for x in range(W):
                e = [x == 0, x == W - 1, y == 0, y == H - 1]
                if edges:
                    for ed in range(4):
                        if e[ed]:
                            for s in range(5):
                                dy, dx = (s - 2, 0) if ed < 2 else (0, s - 2)
                                Y[y, x] += KE[ed, s] @ zp[:, y + 2 + dy, x + 2 + dx]
                if corners:
                    for yb, yo in ((0, e[2]), (1, e[3])):
                        for xb, xo in ((0, e[0]), (1, e[1])):
                            if yo and xo:
                                Y[y, x] += KC[yb, xb] @ zp[:, y + 2, x + 2]
        t, q, xi = Y[..., :32], Y[..., 32:59], Y[..., 64:]
        s_ = np.tanh(t)
        ND = s_ @ WN.T + (xi * s_) @ WD.T
        qp = np.zeros((H + 2, W + 2, 27))
        qp[1:H + 1, 1:W + 1] = q
        L = np.broadcast_to(bL, (H, W, 3)).astype(np.float64)
        for tl in range(9):
            L = L + qp[tl // 3:tl // 3 + H, tl % 3:tl % 3 + W, 3 * tl:3 * tl + 3]
        a[n] = ((L + ND) * outs).transpose(2, 0, 1)
    return a


def _blob(seed):
    return wl.kaiming_blob(seed, in_scale=(2.0, 3.0, 1.0, 0.5, 1.5, 2.5), out_scale=(1.0, 0.5, 2.0),
                           bias_sigma=0.5).astype(np.float64)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 2), (2, 1), (2, 3), (3, 3), (5, 7), (13, 9), (14, 26)])
def test_composite_with_edge_terms_is_the_layered_cell(H, W):
    w = _blob(61)
    z = np.random.default_rng(62 + H * 31 + W).normal(size=(2, 6, H, W))
    ref = oracle.cnn_forward(w, z)
    got = composite_cell(w, z)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_each_correction_is_needed():
    """Without the edge terms the outer ring differs (interior nodes two or
    more from the edge do not); without the corner add-back the four corners
    differ, and beyond them only the nodes whose linear branch reads a
    corner's q (the 2 x 2 block at each corner)."""
    H, W = 9, 11
    w = _blob(63)
    z = np.random.default_rng(64).normal(size=(1, 6, H, W))
    ref = oracle.cnn_forward(w, z)[0]
    scale = np.abs(ref).max()
    bad = np.abs(composite_cell(w, z, edges=False, corners=False)[0] - ref).max(axis=0) > 1e-9 * scale
    ring = np.ones((H, W), bool)
    ring[2:-2, 2:-2] = False
    assert bad[0, :].all() and bad[-1, :].all() and bad[:, 0].all() and bad[:, -1].all()
    assert not bad[~ring].any()
    bad = np.abs(composite_cell(w, z, corners=False)[0] - ref).max(axis=0) > 1e-9 * scale
    corners = np.zeros((H, W), bool)
    corners[0, 0] = corners[0, -1] = corners[-1, 0] = corners[-1, -1] = True
    blocks = np.zeros((H, W), bool)
    for ys in (slice(0, 2), slice(H - 2, H)):
        for xs in (slice(0, 2), slice(W - 2, W)):
            blocks[ys, xs] = True
    assert bad[corners].all() and not bad[~blocks].any()
