/*
 * FP64 CPU oracle for the physics-embedded CNN cell (Sec. 3.2, Eq. 6-7) and
 * its hand-derived backward.
 *
 * TEST INFRASTRUCTURE ONLY.  Loaded by the tests, the package's smoke check
 * and the benchmark's CPU-baseline leg; shares nothing with the CUDA library.
 *
 * The cell ("C-cell"), as read from Eq. 6-7 with the shapes of the CNN
 * inference workload (6 input channels, 32 trunk channels):
 *   zu = in_scale[0:3] * u,  zv = in_scale[3:6] * v   (u = x - X, v: [3][H][W])
 *   phi1 = W1 (*) [zu; 0],   xi1 = W1 (*) [0; zv]     (Eq. 6: one kernel for x and v)
 *   phi  = W2 (*) phi1,      xi  = W2 (*) xi1         (3x3, 32 -> 32, no bias)
 *   L = WL (*) phi + bL                                (Eq. 7 linear branch, 3x3, 32 -> 3)
 *   s = tanh(P phi)                                    (1x1, 32 -> 32)
 *   N = WN s                                           (Eq. 7 nonlinear branch, 1x1, 32 -> 3)
 *   D = WD (xi . s)                                    (Eq. 7 derivative branch, 1x1, 32 -> 3)
 *   a = out_scale * (L + N + D)                        (acceleration, 3 channels)
 * (*) is a 3x3 cross-correlation with zero "same" padding, as
 * torch.nn.functional.conv2d(padding=1) computes it.  The bias appears once,
 * in the linear branch (Sec. 3.2).
 *
 * Weight blob (doubles): W1[32][6][3][3], W2[32][32][3][3], WL[3][32][3][3],
 * bL[3], P[32][32], WN[3][32], WD[3][32], in_scale[6], out_scale[3].  The
 * gradient vector covers the first 13027 entries (the scales are fixed).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { C = 32, CIN = 6, COUT = 3 };
enum {
    OFF_W1 = 0,
    OFF_W2 = OFF_W1 + C * CIN * 9,
    OFF_WL = OFF_W2 + C * C * 9,
    OFF_BL = OFF_WL + COUT * C * 9,
    OFF_P = OFF_BL + COUT,
    OFF_WN = OFF_P + C * C,
    OFF_WD = OFF_WN + COUT * C,
    N_TRAIN = OFF_WD + COUT * C,
    OFF_INS = N_TRAIN,
    OFF_OUTS = OFF_INS + CIN,
    N_BLOB = OFF_OUTS + COUT,
};

int32_t oracle_cnn_param_count(void) { return N_TRAIN; }
int32_t oracle_cnn_blob_count(void) { return N_BLOB; }

/* out[co][y][x] = sum_{ci,ky,kx} w[co][ci][ky][kx] in[ci][y+ky-1][x+kx-1], zero outside. */
static void conv3x3(const double* in, int cin, const double* w, int cout, int H, int W, double* out)
{
    for (int co = 0; co < cout; ++co)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double s = 0.0;
                for (int ci = 0; ci < cin; ++ci)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            const int yy = y + ky - 1, xx = x + kx - 1;
                            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                            s += w[((co * cin + ci) * 3 + ky) * 3 + kx] * in[(ci * H + yy) * W + xx];
                        }
                out[(co * H + y) * W + x] = s;
            }
}

/* Adjoint of conv3x3 with respect to its input: gin += conv3x3^T(gout). */
static void conv3x3_bwd_in(const double* gout, int cout, const double* w, int cin, int H, int W, double* gin)
{
    for (int co = 0; co < cout; ++co)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const double g = gout[(co * H + y) * W + x];
                for (int ci = 0; ci < cin; ++ci)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            const int yy = y + ky - 1, xx = x + kx - 1;
                            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                            gin[(ci * H + yy) * W + xx] += w[((co * cin + ci) * 3 + ky) * 3 + kx] * g;
                        }
            }
}

/* Adjoint of conv3x3 with respect to its weights: gw += d/dw. */
static void conv3x3_bwd_w(const double* gout, int cout, const double* in, int cin, int H, int W, double* gw)
{
    for (int co = 0; co < cout; ++co)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const double g = gout[(co * H + y) * W + x];
                for (int ci = 0; ci < cin; ++ci)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            const int yy = y + ky - 1, xx = x + kx - 1;
                            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                            gw[((co * cin + ci) * 3 + ky) * 3 + kx] += g * in[(ci * H + yy) * W + xx];
                        }
            }
}

/* out[co][p] = sum_ci w[co][ci] in[ci][p] over n pixels. */
static void lin1x1(const double* in, int cin, const double* w, int cout, int n, double* out)
{
    for (int co = 0; co < cout; ++co)
        for (int p = 0; p < n; ++p) {
            double s = 0.0;
            for (int ci = 0; ci < cin; ++ci) s += w[co * cin + ci] * in[ci * n + p];
            out[co * n + p] = s;
        }
}

typedef struct {
    double *zu6, *zv6, *phi1, *xi1, *phi, *xi, *L, *t, *s, *xs, *Nn, *D;
} acts;

static void acts_alloc(acts* A, int n)
{
    A->zu6 = calloc((size_t)CIN * n, sizeof(double));
    A->zv6 = calloc((size_t)CIN * n, sizeof(double));
    A->phi1 = calloc((size_t)C * n, sizeof(double));
    A->xi1 = calloc((size_t)C * n, sizeof(double));
    A->phi = calloc((size_t)C * n, sizeof(double));
    A->xi = calloc((size_t)C * n, sizeof(double));
    A->L = calloc((size_t)COUT * n, sizeof(double));
    A->t = calloc((size_t)C * n, sizeof(double));
    A->s = calloc((size_t)C * n, sizeof(double));
    A->xs = calloc((size_t)C * n, sizeof(double));
    A->Nn = calloc((size_t)COUT * n, sizeof(double));
    A->D = calloc((size_t)COUT * n, sizeof(double));
}

static void acts_free(acts* A)
{
    free(A->zu6); free(A->zv6); free(A->phi1); free(A->xi1); free(A->phi); free(A->xi);
    free(A->L); free(A->t); free(A->s); free(A->xs); free(A->Nn); free(A->D);
}

/* Forward of one sample: z is [6][H][W] (channels u0 u1 u2 v0 v1 v2). */
static void forward_one(const double* wb, int H, int W, const double* z, acts* A, double* a)
{
    const int n = H * W;
    const double* ins = wb + OFF_INS;
    const double* outs = wb + OFF_OUTS;
    for (int k = 0; k < CIN * n; ++k) { A->zu6[k] = 0.0; A->zv6[k] = 0.0; }
    for (int ch = 0; ch < 3; ++ch)
        for (int p = 0; p < n; ++p) {
            A->zu6[ch * n + p] = ins[ch] * z[ch * n + p];
            A->zv6[(ch + 3) * n + p] = ins[ch + 3] * z[(ch + 3) * n + p];
        }
    conv3x3(A->zu6, CIN, wb + OFF_W1, C, H, W, A->phi1);   /* Eq. 6, from x */
    conv3x3(A->zv6, CIN, wb + OFF_W1, C, H, W, A->xi1);    /* Eq. 6, from v */
    conv3x3(A->phi1, C, wb + OFF_W2, C, H, W, A->phi);
    conv3x3(A->xi1, C, wb + OFF_W2, C, H, W, A->xi);
    conv3x3(A->phi, C, wb + OFF_WL, COUT, H, W, A->L);     /* Eq. 7, linear */
    for (int co = 0; co < COUT; ++co)
        for (int p = 0; p < n; ++p) A->L[co * n + p] += wb[OFF_BL + co];
    lin1x1(A->phi, C, wb + OFF_P, C, n, A->t);
    for (int k = 0; k < C * n; ++k) {
        A->s[k] = tanh(A->t[k]);
        A->xs[k] = A->xi[k] * A->s[k];
    }
    lin1x1(A->s, C, wb + OFF_WN, COUT, n, A->Nn);            /* Eq. 7, nonlinear */
    lin1x1(A->xs, C, wb + OFF_WD, COUT, n, A->D);            /* Eq. 7, derivative */
    for (int co = 0; co < COUT; ++co)
        for (int p = 0; p < n; ++p)
            a[co * n + p] = outs[co] * (A->L[co * n + p] + A->Nn[co * n + p] + A->D[co * n + p]);
}

/* a[N][3][H][W] = cell(z[N][6][H][W]). */
void oracle_cnn_forward(const double* wb, int32_t N, int32_t H, int32_t W, const double* z, double* a)
{
    const int n = H * W;
    acts A;
    acts_alloc(&A, n);
    for (int b = 0; b < N; ++b) forward_one(wb, H, W, z + (size_t)b * CIN * n, &A, a + (size_t)b * COUT * n);
    acts_free(&A);
}

/* Backward: given ga[N][3][H][W] = dLoss/da, accumulate nothing and write
 * gw[13027] = dLoss/dw and (if gz != NULL) gz[N][6][H][W] = dLoss/dz. */
void oracle_cnn_backward(const double* wb, int32_t N, int32_t H, int32_t W, const double* z,
                         const double* ga, double* gw, double* gz)
{
    const int n = H * W;
    acts A;
    acts_alloc(&A, n);
    double* a = calloc((size_t)COUT * n, sizeof(double));
    double* gy = calloc((size_t)COUT * n, sizeof(double));
    double* gphi = calloc((size_t)C * n, sizeof(double));
    double* gxi = calloc((size_t)C * n, sizeof(double));
    double* gs = calloc((size_t)C * n, sizeof(double));
    double* gxs = calloc((size_t)C * n, sizeof(double));
    double* gt = calloc((size_t)C * n, sizeof(double));
    double* gphi1 = calloc((size_t)C * n, sizeof(double));
    double* gxi1 = calloc((size_t)C * n, sizeof(double));
    double* gzu6 = calloc((size_t)CIN * n, sizeof(double));
    double* gzv6 = calloc((size_t)CIN * n, sizeof(double));
    const double* outs = wb + OFF_OUTS;
    const double* ins = wb + OFF_INS;
    const double* P = wb + OFF_P;
    const double* WN = wb + OFF_WN;
    const double* WD = wb + OFF_WD;
    for (int k = 0; k < N_TRAIN; ++k) gw[k] = 0.0;

    for (int b = 0; b < N; ++b) {
        const double* zb = z + (size_t)b * CIN * n;
        const double* gab = ga + (size_t)b * COUT * n;
        forward_one(wb, H, W, zb, &A, a);
        memset(gphi, 0, sizeof(double) * C * n);
        memset(gxi, 0, sizeof(double) * C * n);
        memset(gs, 0, sizeof(double) * C * n);
        memset(gphi1, 0, sizeof(double) * C * n);
        memset(gxi1, 0, sizeof(double) * C * n);
        memset(gzu6, 0, sizeof(double) * CIN * n);
        memset(gzv6, 0, sizeof(double) * CIN * n);

        /* a = out_scale (L + N + D) */
        for (int co = 0; co < COUT; ++co)
            for (int p = 0; p < n; ++p) gy[co * n + p] = outs[co] * gab[co * n + p];
        /* L = WL (*) phi + bL */
        for (int co = 0; co < COUT; ++co)
            for (int p = 0; p < n; ++p) gw[OFF_BL + co] += gy[co * n + p];
        conv3x3_bwd_w(gy, COUT, A.phi, C, H, W, gw + OFF_WL);
        conv3x3_bwd_in(gy, COUT, wb + OFF_WL, C, H, W, gphi);
        /* N = WN s,  D = WD (xi . s) */
        for (int co = 0; co < COUT; ++co)
            for (int c = 0; c < C; ++c)
                for (int p = 0; p < n; ++p) {
                    gw[OFF_WN + co * C + c] += gy[co * n + p] * A.s[c * n + p];
                    gw[OFF_WD + co * C + c] += gy[co * n + p] * A.xs[c * n + p];
                }
        for (int c = 0; c < C; ++c)
            for (int p = 0; p < n; ++p) {
                double gsn = 0.0, gxsn = 0.0;
                for (int co = 0; co < COUT; ++co) {
                    gsn += WN[co * C + c] * gy[co * n + p];
                    gxsn += WD[co * C + c] * gy[co * n + p];
                }
                gxs[c * n + p] = gxsn;
                gs[c * n + p] = gsn + gxsn * A.xi[c * n + p];
                gxi[c * n + p] += gxsn * A.s[c * n + p];
            }
        /* s = tanh(t), t = P phi */
        for (int k = 0; k < C * n; ++k) gt[k] = gs[k] * (1.0 - A.s[k] * A.s[k]);
        for (int c = 0; c < C; ++c)
            for (int c2 = 0; c2 < C; ++c2)
                for (int p = 0; p < n; ++p) {
                    gw[OFF_P + c * C + c2] += gt[c * n + p] * A.phi[c2 * n + p];
                    gphi[c2 * n + p] += P[c * C + c2] * gt[c * n + p];
                }
        /* phi = W2 (*) phi1, xi = W2 (*) xi1 */
        conv3x3_bwd_w(gphi, C, A.phi1, C, H, W, gw + OFF_W2);
        conv3x3_bwd_w(gxi, C, A.xi1, C, H, W, gw + OFF_W2);
        conv3x3_bwd_in(gphi, C, wb + OFF_W2, C, H, W, gphi1);
        conv3x3_bwd_in(gxi, C, wb + OFF_W2, C, H, W, gxi1);
        /* phi1 = W1 (*) [zu; 0], xi1 = W1 (*) [0; zv] */
        conv3x3_bwd_w(gphi1, C, A.zu6, CIN, H, W, gw + OFF_W1);
        conv3x3_bwd_w(gxi1, C, A.zv6, CIN, H, W, gw + OFF_W1);
        if (gz) {
            conv3x3_bwd_in(gphi1, C, wb + OFF_W1, CIN, H, W, gzu6);
            conv3x3_bwd_in(gxi1, C, wb + OFF_W1, CIN, H, W, gzv6);
            double* gzb = gz + (size_t)b * CIN * n;
            for (int ch = 0; ch < 3; ++ch)
                for (int p = 0; p < n; ++p) {
                    gzb[ch * n + p] = ins[ch] * gzu6[ch * n + p];
                    gzb[(ch + 3) * n + p] = ins[ch + 3] * gzv6[(ch + 3) * n + p];
                }
        }
    }
    acts_free(&A);
    free(a); free(gy); free(gphi); free(gxi); free(gs); free(gxs); free(gt);
    free(gphi1); free(gxi1); free(gzu6); free(gzv6);
}
