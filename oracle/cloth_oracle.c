/*
 * FP64 CPU oracle for the regular-grid mass-spring cloth (Sec. 3.1, Eq. 1-5).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU plain step computes.  It is compiled into
 * oracle/liboracle.so and may be loaded only by the tests, by the package's
 * smoke check and by the CPU-baseline leg of the benchmark.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Layout: one cloth of rows x cols nodes; node (r, c) has index r*cols + c and
 * rest position X = (c*h, r*h, 0).  Positions and velocities are arrays
 * [rows][cols][3] of doubles.
 *
 * Readings of the paper (where it is silent or ambiguous):
 *  - x_ij = x_i - x_j and v_ij = v_i - v_j (Eq. 1, 2); the leading minus then
 *    makes a stretched spring pull i towards j.
 *  - "E" of Eq. 1 is a per-type spring stiffness k (N/m): structural springs
 *    to the 4 cardinal neighbours, shear springs to the 4 diagonal ones, bend
 *    springs to the 4 nodes two apart in the cardinal directions (Sec. 3.1,
 *    13-point stencil).  Rest lengths come from the undeformed lattice:
 *    h, sqrt(2) h, 2 h.
 *  - Eq. 3 is scaled by 1/4, so that a flat interior node receives p h^2,
 *    i.e. the pressure times its lumped area.  The 4 ordered pairs are
 *    (E,N), (N,W), (W,S), (S,E), which gives a flat cloth the normal +z; a
 *    pair contributes only when both of its nodes exist.
 *  - The constraint operator C of Eq. 5 sets the velocity of pinned nodes
 *    to the velocity of the object they move with (zero for a fixed node,
 *    the Dirichlet case) before the position update; M^-1 is the inverse
 *    lumped (uniform) mass.
 *  - Sphere contact (intersection elimination, Sec. 3.1) is a projection of
 *    the updated position onto the sphere surface, applied after the
 *    update.  The velocity then either stops (the ball of Sec. 3.2.2 that
 *    absorbs the bounce and whose friction prevents relative motion; a
 *    negative friction coefficient) or, for a coefficient mu >= 0, loses
 *    its approaching normal part and Coulomb friction reduces its
 *    tangential part by at most mu times that normal part.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t rows, cols;
    double h;                          /* lattice spacing, m                     */
    double m;                          /* node mass, kg                          */
    double k_struct, k_shear, k_bend;  /* spring stiffness per type, N/m (Eq. 1) */
    double mu;                         /* spring-axis damping (Eq. 2)            */
    double drag;                       /* air drag d (Eq. 4)                     */
    double p;                          /* pressure (Eq. 3)                       */
    double g[3];                       /* gravity acceleration (Eq. 4)           */
    double dt;                         /* time step (Eq. 5)                      */
    int32_t sphere_on;                 /* sphere contact enabled                 */
    double sphere_c[3];
    double sphere_r;
    double sphere_mu;                  /* < 0: contact sticks; else Coulomb mu   */
    double pin_v[3];                   /* velocity of the pinned nodes, m/s      */
} oracle_cloth;

/* The 13-point stencil: the centre plus these 12 neighbour offsets (dr, dc).
 * 0-3 structural (E, N, W, S), 4-7 shear (NE, NW, SW, SE), 8-11 bend. */
static const int OFF[12][2] = {
    {0, 1}, {1, 0}, {0, -1}, {-1, 0},
    {1, 1}, {1, -1}, {-1, -1}, {-1, 1},
    {0, 2}, {2, 0}, {0, -2}, {-2, 0},
};

static double spring_k(const oracle_cloth* c, int s)
{
    if (s < 4) return c->k_struct;
    if (s < 8) return c->k_shear;
    return c->k_bend;
}

static double spring_rest(const oracle_cloth* c, int s)
{
    if (s < 4) return c->h;
    if (s < 8) return sqrt(2.0) * c->h;
    return 2.0 * c->h;
}

static int in_grid(const oracle_cloth* c, int r, int col)
{
    return r >= 0 && r < c->rows && col >= 0 && col < c->cols;
}

/* Bit s of mask[i] is set iff neighbour s of node i lies in the grid, i.e.
 * iff the spring (i, i + OFF[s]) exists. */
void oracle_neighbor_mask(int32_t rows, int32_t cols, uint16_t* mask)
{
    oracle_cloth c;
    memset(&c, 0, sizeof c);
    c.rows = rows;
    c.cols = cols;
    for (int r = 0; r < rows; ++r)
        for (int col = 0; col < cols; ++col) {
            uint16_t b = 0;
            for (int s = 0; s < 12; ++s)
                if (in_grid(&c, r + OFF[s][0], col + OFF[s][1])) b |= (uint16_t)(1u << s);
            mask[r * cols + col] = b;
        }
}

/* Number of springs of each type, counting every (i, j) pair once. */
void oracle_spring_counts(int32_t rows, int32_t cols, int64_t counts[3])
{
    int64_t twice[3] = {0, 0, 0};
    oracle_cloth c;
    memset(&c, 0, sizeof c);
    c.rows = rows;
    c.cols = cols;
    for (int r = 0; r < rows; ++r)
        for (int col = 0; col < cols; ++col)
            for (int s = 0; s < 12; ++s)
                if (in_grid(&c, r + OFF[s][0], col + OFF[s][1])) twice[s / 4] += 1;
    for (int t = 0; t < 3; ++t) counts[t] = twice[t] / 2;
}

/* Internal spring forces, Eq. 1 (elastic) + Eq. 2 (spring-axis damping). */
void oracle_internal_force(const oracle_cloth* c, const double* x, const double* v, double* f)
{
    for (int r = 0; r < c->rows; ++r)
        for (int col = 0; col < c->cols; ++col) {
            const int i = r * c->cols + col;
            double fi[3] = {0.0, 0.0, 0.0};
            for (int s = 0; s < 12; ++s) {
                const int rj = r + OFF[s][0], cj = col + OFF[s][1];
                if (!in_grid(c, rj, cj)) continue;
                const int j = rj * c->cols + cj;
                double xij[3], vij[3];
                for (int a = 0; a < 3; ++a) {
                    xij[a] = x[3 * i + a] - x[3 * j + a];
                    vij[a] = v[3 * i + a] - v[3 * j + a];
                }
                const double len = sqrt(xij[0] * xij[0] + xij[1] * xij[1] + xij[2] * xij[2]);
                double xhat[3];
                for (int a = 0; a < 3; ++a) xhat[a] = xij[a] / len;
                const double k = spring_k(c, s), L = spring_rest(c, s);
                const double vproj = vij[0] * xhat[0] + vij[1] * xhat[1] + vij[2] * xhat[2];
                for (int a = 0; a < 3; ++a) {
                    fi[a] += -k * xhat[a] * (len - L);   /* Eq. 1 */
                    fi[a] += -c->mu * vproj * xhat[a];   /* Eq. 2 */
                }
            }
            for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];
        }
}

static void cross(const double* a, const double* b, double* out)
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Pressure force, Eq. 3 scaled by 1/4, over the ordered cardinal pairs
 * (E,N), (N,W), (W,S), (S,E); x_ij = x_i - x_j. */
void oracle_pressure_force(const oracle_cloth* c, const double* x, double* f)
{
    static const int PAIR[4][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}}; /* indices into OFF */
    for (int r = 0; r < c->rows; ++r)
        for (int col = 0; col < c->cols; ++col) {
            const int i = r * c->cols + col;
            double fi[3] = {0.0, 0.0, 0.0};
            for (int q = 0; q < 4; ++q) {
                const int s1 = PAIR[q][0], s2 = PAIR[q][1];
                const int r1 = r + OFF[s1][0], c1 = col + OFF[s1][1];
                const int r2 = r + OFF[s2][0], c2 = col + OFF[s2][1];
                if (!in_grid(c, r1, c1) || !in_grid(c, r2, c2)) continue;
                const int j1 = r1 * c->cols + c1, j2 = r2 * c->cols + c2;
                double x1[3], x2[3], cr[3];
                for (int a = 0; a < 3; ++a) {
                    x1[a] = x[3 * i + a] - x[3 * j1 + a];
                    x2[a] = x[3 * i + a] - x[3 * j2 + a];
                }
                cross(x1, x2, cr);
                for (int a = 0; a < 3; ++a) fi[a] += 0.25 * c->p * cr[a];
            }
            for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];
        }
}

/* Vector-Jacobian product of the pressure force (Eq. 3, 1/4 reading) with
 * respect to the positions: gx = (d f_p / d x)^T gf.  For one pair term
 * T = a x b with a = x_i - x_j1, b = x_i - x_j2 and cotangent G:
 * d(G.T)/da = b x G and d(G.T)/db = G x a. */
void oracle_pressure_vjp(const oracle_cloth* c, const double* x, const double* gf, double* gx)
{
    static const int PAIR[4][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}};
    const int n = c->rows * c->cols;
    for (int k = 0; k < 3 * n; ++k) gx[k] = 0.0;
    for (int r = 0; r < c->rows; ++r)
        for (int col = 0; col < c->cols; ++col) {
            const int i = r * c->cols + col;
            for (int q = 0; q < 4; ++q) {
                const int s1 = PAIR[q][0], s2 = PAIR[q][1];
                const int r1 = r + OFF[s1][0], c1 = col + OFF[s1][1];
                const int r2 = r + OFF[s2][0], c2 = col + OFF[s2][1];
                if (!in_grid(c, r1, c1) || !in_grid(c, r2, c2)) continue;
                const int j1 = r1 * c->cols + c1, j2 = r2 * c->cols + c2;
                double a[3], b[3], G[3], ga[3], gb[3];
                for (int k = 0; k < 3; ++k) {
                    a[k] = x[3 * i + k] - x[3 * j1 + k];
                    b[k] = x[3 * i + k] - x[3 * j2 + k];
                    G[k] = 0.25 * c->p * gf[3 * i + k];
                }
                cross(b, G, ga);
                cross(G, a, gb);
                for (int k = 0; k < 3; ++k) {
                    gx[3 * i + k] += ga[k] + gb[k];
                    gx[3 * j1 + k] -= ga[k];
                    gx[3 * j2 + k] -= gb[k];
                }
            }
        }
}

/* Gravity and air drag, Eq. 4. */
void oracle_external_force(const oracle_cloth* c, const double* v, double* f)
{
    const int n = c->rows * c->cols;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) f[3 * i + a] = c->m * c->g[a] - c->drag * v[3 * i + a];
}

/* Total force on every node: Eq. 1 + 2 + 3 + 4. */
void oracle_total_force(const oracle_cloth* c, const double* x, const double* v, double* f)
{
    const int n = c->rows * c->cols;
    double* tmp = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    oracle_internal_force(c, x, v, f);
    oracle_pressure_force(c, x, tmp);
    for (int k = 0; k < 3 * n; ++k) f[k] += tmp[k];
    oracle_external_force(c, v, tmp);
    for (int k = 0; k < 3 * n; ++k) f[k] += tmp[k];
    free(tmp);
}

/* Sphere contact: a node found inside the sphere is moved to the nearest
 * point of its surface.  With sphere_mu < 0 it stops.  Otherwise, with n
 * the outward normal, v_n = v . n and v_t = v - v_n n: the approaching part
 * j = max(-v_n, 0) is absorbed and friction takes min(|v_t|, mu j) off the
 * tangential speed. */
static void sphere_project(const oracle_cloth* c, double* x, double* v)
{
    if (!c->sphere_on) return;
    const int n = c->rows * c->cols;
    for (int i = 0; i < n; ++i) {
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = x[3 * i + a] - c->sphere_c[a];
        const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (len < c->sphere_r && len > 0.0) {
            double nrm[3], vn = 0.0;
            for (int a = 0; a < 3; ++a) {
                nrm[a] = d[a] / len;
                x[3 * i + a] = c->sphere_c[a] + c->sphere_r * nrm[a];
                vn += v[3 * i + a] * nrm[a];
            }
            if (c->sphere_mu < 0.0) {
                for (int a = 0; a < 3; ++a) v[3 * i + a] = 0.0;
                continue;
            }
            double vt[3], tl2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                vt[a] = v[3 * i + a] - vn * nrm[a];
                tl2 += vt[a] * vt[a];
            }
            const double tl = sqrt(tl2);
            const double j = vn < 0.0 ? -vn : 0.0;
            const double keep = tl > c->sphere_mu * j ? 1.0 - c->sphere_mu * j / tl : 0.0;
            const double vn_out = vn > 0.0 ? vn : 0.0;
            for (int a = 0; a < 3; ++a) v[3 * i + a] = vn_out * nrm[a] + keep * vt[a];
        }
    }
}

/* The update of Eq. 5 for a given acceleration acc (m/s^2, per node):
 *   v <- C(v + dt acc);  x <- x + dt v;  then sphere contact,
 * where C sets pinned velocities (pinned[i] != 0) to pin_v. */
void oracle_update(const oracle_cloth* c, const uint8_t* pinned, const double* acc, double* x, double* v)
{
    const int n = c->rows * c->cols;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double vn = v[3 * i + a] + c->dt * acc[3 * i + a];
            if (pinned && pinned[i]) vn = c->pin_v[a];
            v[3 * i + a] = vn;
            x[3 * i + a] += c->dt * vn;
        }
    sphere_project(c, x, v);
}

/* Advance `steps` semi-implicit Euler steps in place (Eq. 5) with the
 * plain step's acceleration f / m (oracle_update).  pinned[i] != 0 marks a
 * node that moves with pin_v (held in place when pin_v = 0). */
void oracle_step(const oracle_cloth* c, const uint8_t* pinned, double* x, double* v, int32_t steps)
{
    const int n = c->rows * c->cols;
    double* f = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    for (int t = 0; t < steps; ++t) {
        oracle_total_force(c, x, v, f);
        for (int k = 0; k < 3 * n; ++k) f[k] /= c->m;
        oracle_update(c, pinned, f, x, v);
    }
    free(f);
}

/* Total mechanical energy: kinetic + elastic (sum over springs, each once)
 * + gravitational (-m g . x). */
double oracle_energy(const oracle_cloth* c, const double* x, const double* v)
{
    double ke = 0.0, pe = 0.0, pg = 0.0;
    for (int r = 0; r < c->rows; ++r)
        for (int col = 0; col < c->cols; ++col) {
            const int i = r * c->cols + col;
            for (int a = 0; a < 3; ++a) {
                ke += 0.5 * c->m * v[3 * i + a] * v[3 * i + a];
                pg -= c->m * c->g[a] * x[3 * i + a];
            }
            for (int s = 0; s < 12; ++s) {
                const int rj = r + OFF[s][0], cj = col + OFF[s][1];
                if (!in_grid(c, rj, cj)) continue;
                const int j = rj * c->cols + cj;
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double d = x[3 * i + a] - x[3 * j + a];
                    d2 += d * d;
                }
                const double ext = sqrt(d2) - spring_rest(c, s);
                pe += 0.5 * 0.5 * spring_k(c, s) * ext * ext; /* each spring seen from both ends */
            }
        }
    return ke + pe + pg;
}
