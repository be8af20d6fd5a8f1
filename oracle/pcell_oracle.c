/* FP64 oracle of the physics-embedded cell read literally (test
 * infrastructure only): Sec. 3.2, Eq. 6-7 and Fig. 1.
 *
 * Eq. 6: the same 2D kernels act on every coordinate of x and of v (the
 * isotropy assumption), and channel c is a frozen filter that takes the
 * correlation of the node with one of the 12 neighbours of the 13-point
 * stencil of Sec. 3.1: the difference  phi_c = x_j - x_i  (xi_c = v_j - v_i
 * for the velocity), with the 8 taps of a 3x3 kernel for the structural and
 * shear neighbours and the 4 cardinal taps of a dilation-2 3x3 kernel for
 * the bending neighbours.  A neighbour outside the grid contributes no
 * channel (no spring exists there).
 *
 * Eq. 7, per coordinate k and node i, summed over the channels c:
 *   L = sum_c w_L[c] phi_c,k + b_L[k]            (one bias per coordinate)
 *   N = sum_c w_N[c] sigma(phi_c,k)
 *   D = sum_c w_D[c] xi_c,k sigma(phi_c,k)
 *   a = L + N + D
 * with sigma the inverse square root unit sigma(z) = z / sqrt(1 + alpha z^2).
 *
 * Parameter blob (40 doubles): w_L[12], w_N[12], w_D[12], b_L[3], alpha.
 * Channel order (row offset dy, column offset dx):
 *   E (0,1), W (0,-1), N (1,0), S (-1,0), NE (1,1), NW (1,-1), SE (-1,1),
 *   SW (-1,-1), E2 (0,2), W2 (0,-2), N2 (2,0), S2 (-2,0).
 * Arrays are row-major [rows][cols][3].
 */
#include <math.h>
#include <stdint.h>

static const int kDy[12] = {0, 0, 1, -1, 1, 1, -1, -1, 0, 0, 2, -2};
static const int kDx[12] = {1, -1, 0, 0, 1, -1, 1, -1, 2, -2, 0, 0};

void oracle_pcell_accel(int32_t rows, int32_t cols, const double* w, const double* x, const double* v, double* a)
{
    const double* wL = w;
    const double* wN = w + 12;
    const double* wD = w + 24;
    const double* bL = w + 36;
    const double alpha = w[39];
    for (int r = 0; r < rows; ++r) {
        for (int c = 0; c < cols; ++c) {
            const int64_t i = (int64_t)r * cols + c;
            for (int k = 0; k < 3; ++k) {
                double acc = bL[k];
                for (int ch = 0; ch < 12; ++ch) {
                    const int rr = r + kDy[ch], cc = c + kDx[ch];
                    if (rr < 0 || rr >= rows || cc < 0 || cc >= cols) continue;
                    const int64_t j = (int64_t)rr * cols + cc;
                    const double phi = x[3 * j + k] - x[3 * i + k];
                    const double xi = v[3 * j + k] - v[3 * i + k];
                    const double s = phi / sqrt(1.0 + alpha * phi * phi);
                    acc += wL[ch] * phi + wN[ch] * s + wD[ch] * xi * s;
                }
                a[3 * i + k] = acc;
            }
        }
    }
}

/* Backward of oracle_pcell_accel for a cotangent ga [rows][cols][3]: the
 * gradient of sum(ga . a) with respect to the 39 trainable parameters
 * (w_L, w_N, w_D, b_L; alpha is a fixed hyper-parameter) added to gw, and
 * with respect to x and v added to gx, gv.  Per channel term
 * t = w_L phi + w_N s + w_D xi s, s = phi (1 + alpha phi^2)^(-1/2):
 *   dt/dphi = w_L + (w_N + w_D xi) (1 + alpha phi^2)^(-3/2),
 *   dt/dxi = w_D s,  and phi = x_j - x_i, xi = v_j - v_i. */
void oracle_pcell_backward(int32_t rows, int32_t cols, const double* w, const double* x, const double* v,
                           const double* ga, double* gw, double* gx, double* gv)
{
    const double* wL = w;
    const double* wN = w + 12;
    const double* wD = w + 24;
    const double alpha = w[39];
    for (int r = 0; r < rows; ++r) {
        for (int c = 0; c < cols; ++c) {
            const int64_t i = (int64_t)r * cols + c;
            for (int k = 0; k < 3; ++k) {
                const double g = ga[3 * i + k];
                gw[36 + k] += g;
                for (int ch = 0; ch < 12; ++ch) {
                    const int rr = r + kDy[ch], cc = c + kDx[ch];
                    if (rr < 0 || rr >= rows || cc < 0 || cc >= cols) continue;
                    const int64_t j = (int64_t)rr * cols + cc;
                    const double phi = x[3 * j + k] - x[3 * i + k];
                    const double xi = v[3 * j + k] - v[3 * i + k];
                    const double q = 1.0 + alpha * phi * phi;
                    const double s = phi / sqrt(q);
                    const double ds = 1.0 / (q * sqrt(q));
                    gw[ch] += g * phi;
                    gw[12 + ch] += g * s;
                    gw[24 + ch] += g * xi * s;
                    const double gphi = g * (wL[ch] + (wN[ch] + wD[ch] * xi) * ds);
                    const double gxi = g * wD[ch] * s;
                    gx[3 * j + k] += gphi;
                    gx[3 * i + k] -= gphi;
                    gv[3 * j + k] += gxi;
                    gv[3 * i + k] -= gxi;
                }
            }
        }
    }
}
