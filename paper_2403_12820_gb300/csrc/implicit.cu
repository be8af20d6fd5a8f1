// Implicit plain step: linearised backward Euler (Sec. 3.1 names implicit
// integration as the stable choice for large time steps; Sec. 5 lists it as
// the comparison for a larger-step cell).  One Newton step of
// v' = v + h M^-1 f(x + h v', v') with the elastic springs (Eq. 1) and the
// air drag (Eq. 4) implicit, the rest (Eq. 2 damping, Eq. 3 pressure,
// gravity) explicit:
//   (m + h d) dv - h^2 K dv = h f(x, v) + h^2 K v,   v' = C(v + dv),
//   x' = x + h v', sphere contact,
// K = df/dx of the springs; per spring (i, j), d = x_j - x_i, l = |d|,
// n = d / l: K_s = k [n n^T + c (I - n n^T)], c = max(0, 1 - L / l) (the
// transverse part clamped under compression keeps the matrix SPD), and
// (K w)_i = sum_j K_s (w_j - w_i).
//
// The system is solved matrix-free by conjugate gradients, per cloth (each
// cloth has its own step lengths), a fixed number of iterations.  Pinned
// nodes take dv = pin_v - v and are filtered out of the residual and the
// search direction.  Vectors (dv, r, p, A p) use the state buffers' plane
// layout (planes 0-2); dot products are summed per block and then over the
// blocks in a fixed order, so a step is bitwise reproducible.
#include "cloth_internal.cuh"

namespace cloth {
namespace {

constexpr int TB = 256;

struct ImplArgs {
    const ClothDesc* desc;
    const uint32_t* pinmask;
    const float* state;      // current state (u, v planes)
    const float* f_abi;      // explicit forces, packed ABI layout [node][3]
    float* dv;
    float* r;
    float* p;
    float* ap;
    float* part;             // [B][gx] block partial sums
    float* rr;               // [B]: r . r
    float* rr_new;           // [B]
    float* pap;              // [B]: p . A p
    const int32_t* blk;      // [B + 1]: first block of each cloth (blocks of TB nodes)
    int B;
    int gx;                  // partial sums per cloth (the most blocks of one cloth)
    float h;                 // the step
};

// The cloth b of this block and the block's index k within the cloth.
__device__ __forceinline__ void locate(const ImplArgs& A, int& b, int& k)
{
    const int x = (int)blockIdx.x;
    int lo = 0, hi = A.B - 1;
    while (lo < hi) {   // last b with blk[b] <= x
        const int mid = (lo + hi + 1) >> 1;
        if (A.blk[mid] <= x) lo = mid; else hi = mid - 1;
    }
    b = lo;
    k = x - A.blk[lo];
}

__device__ __forceinline__ bool pinned_at(const ClothDesc& D, const uint32_t* pm, int r, int c)
{
    return (pm[D.pin_off + (int64_t)r * D.pin_wpr + (c >> 5)] >> (c & 31)) & 1u;
}

// 12 stencil neighbours: row, column offset; spring type (0 struct, 1 shear, 2 bend)
__device__ __forceinline__ int nb_dy(int s) { return s == 1 || s == 4 || s == 5 ? 1 : (s == 3 || s == 6 || s == 7 ? -1 : (s == 9 ? 2 : (s == 11 ? -2 : 0))); }
__device__ __forceinline__ int nb_dx(int s) { return s == 0 || s == 4 || s == 7 ? 1 : (s == 2 || s == 5 || s == 6 ? -1 : (s == 8 ? 2 : (s == 10 ? -2 : 0))); }
__device__ __forceinline__ int nb_type(int s) { return s < 4 ? 0 : (s < 8 ? 1 : 2); }

// sum_j K_s(ij) (w_j - w_i) at node (r, c) of a cloth whose u planes start
// at U (plane stride ps, offsets within the cloth in 32 bits); w is read
// through wat(offset, row, column, w)
template <class W>
__device__ __forceinline__ void kw(const ClothDesc& D, const float* __restrict__ U, int ps, int r, int c, W wat,
                                   float (&out)[3])
{
    const int rows = D.rows, cols = D.cols, pitch = D.pitch;
    const float h = D.h, kst = D.k_struct, ksh = D.k_shear, kbe = D.k_bend;
    const int oi = r * pitch + col_pos(c);
    const float ui[3] = {U[oi], U[oi + ps], U[oi + 2 * ps]};
    float wi[3];
    wat(oi, r, c, wi);
    out[0] = out[1] = out[2] = 0.f;
#pragma unroll
    for (int s = 0; s < 12; ++s) {
        const int dy = nb_dy(s), dx = nb_dx(s), rj = r + dy, cj = c + dx;
        if (rj < 0 || rj >= rows || cj < 0 || cj >= cols) continue;
        const int t = nb_type(s);
        const float k = t == 0 ? kst : (t == 1 ? ksh : kbe);
        const float L = t == 0 ? h : (t == 1 ? 1.41421356237309515f * h : 2.f * h);
        const int oj = rj * pitch + col_pos(cj);
        const float d0 = fmaf((float)dx, h, U[oj] - ui[0]);
        const float d1 = fmaf((float)dy, h, U[oj + ps] - ui[1]);
        const float d2 = U[oj + 2 * ps] - ui[2];
        const float rl = rsqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
        const float n0 = d0 * rl, n1 = d1 * rl, n2 = d2 * rl;
        const float cc = fmaxf(0.f, 1.f - L * rl);
        float wj[3];
        wat(oj, rj, cj, wj);
        const float e0 = wj[0] - wi[0], e1 = wj[1] - wi[1], e2 = wj[2] - wi[2];
        const float ne = fmaf(n0, e0, fmaf(n1, e1, n2 * e2));
        // k [c e + (1 - c) (n . e) n]
        const float a = k * cc, b = k * (1.f - cc) * ne;
        out[0] = fmaf(a, e0, fmaf(b, n0, out[0]));
        out[1] = fmaf(a, e1, fmaf(b, n1, out[1]));
        out[2] = fmaf(a, e2, fmaf(b, n2, out[2]));
    }
}

__device__ __forceinline__ float block_sum(float v, float* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < TB / 32; ++w) s += red[w];
    return s;   // valid in thread 0
}

// dv0 (0 free, pin_v - v pinned), r0 = b - A dv0 (free nodes), p0 = r0,
// block partials of r0 . r0
__global__ void __launch_bounds__(TB) impl_rhs_kernel(ImplArgs A)
{
    __shared__ float red[TB / 32];
    int b, kb;
    locate(A, b, kb);
    const ClothDesc& D = A.desc[b];
    const int n = D.rows * D.cols, ps = (int)D.plane_stride;
    const int i = kb * TB + (int)threadIdx.x;
    float rr = 0.f;
    if (i < n) {
        const int r = i / D.cols, c = i % D.cols;
        const int64_t o = D.plane_off + r * D.pitch + col_pos(c);
        const float* U = A.state + D.plane_off;
        const float* V = U + 3 * D.plane_stride;
        auto vat = [&](int q, int, int, float (&w)[3]) { w[0] = V[q]; w[1] = V[q + ps]; w[2] = V[q + 2 * ps]; };
        auto dv0 = [&](int q, int rr_, int cc_, float (&w)[3]) {
            float v[3];
            vat(q, rr_, cc_, v);
            const bool pj = pinned_at(D, A.pinmask, rr_, cc_);
#pragma unroll
            for (int k = 0; k < 3; ++k) w[k] = pj ? pin_v(D, k) - v[k] : 0.f;
        };
        const bool pi = pinned_at(D, A.pinmask, r, c);
        float kv[3], kd[3], d0[3];
        kw(D, U, ps, r, c, vat, kv);
        kw(D, U, ps, r, c, dv0, kd);
        dv0(r * D.pitch + col_pos(c), r, c, d0);
        const float hh = A.h * A.h, md = D.m + A.h * D.drag;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float f = A.f_abi[(D.abi_off + i) * 3 + k];
            const float bk = fmaf(A.h, f, hh * kv[k]);
            const float ak = fmaf(md, d0[k], -hh * kd[k]);
            const float rk = pi ? 0.f : bk - ak;
            A.dv[o + k * D.plane_stride] = d0[k];
            A.r[o + k * D.plane_stride] = rk;
            A.p[o + k * D.plane_stride] = rk;
            rr = fmaf(rk, rk, rr);
        }
    }
    const float s = block_sum(rr, red);
    if (threadIdx.x == 0) A.part[(int64_t)b * A.gx + kb] = s;
}

// A p (filtered: 0 at pinned nodes) and block partials of p . A p
__global__ void __launch_bounds__(TB) impl_matvec_kernel(ImplArgs A)
{
    __shared__ float red[TB / 32];
    int b, kb;
    locate(A, b, kb);
    const ClothDesc& D = A.desc[b];
    const int n = D.rows * D.cols, ps = (int)D.plane_stride;
    const int i = kb * TB + (int)threadIdx.x;
    float pap = 0.f;
    if (i < n) {
        const int r = i / D.cols, c = i % D.cols;
        const int oi = r * D.pitch + col_pos(c);
        const int64_t o = D.plane_off + oi;
        const float* P = A.p + D.plane_off;
        auto pat = [&](int q, int, int, float (&w)[3]) { w[0] = P[q]; w[1] = P[q + ps]; w[2] = P[q + 2 * ps]; };
        const bool pi = pinned_at(D, A.pinmask, r, c);
        float kp[3], pv[3];
        kw(D, A.state + D.plane_off, ps, r, c, pat, kp);
        pat(oi, r, c, pv);
        const float hh = A.h * A.h, md = D.m + A.h * D.drag;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float ak = pi ? 0.f : fmaf(md, pv[k], -hh * kp[k]);
            A.ap[o + k * D.plane_stride] = ak;
            pap = fmaf(pv[k], ak, pap);
        }
    }
    const float s = block_sum(pap, red);
    if (threadIdx.x == 0) A.part[(int64_t)b * A.gx + kb] = s;
}

// out[b] = sum of cloth b's block partials, in block order (one warp per cloth)
__global__ void impl_reduce_kernel(const ClothDesc* __restrict__ desc, const float* __restrict__ part, int gx,
                                   float* __restrict__ out)
{
    const int b = blockIdx.x, lane = threadIdx.x;
    const ClothDesc& D = desc[b];
    const int nb = (int)(((int64_t)D.rows * D.cols + TB - 1) / TB);
    float s = 0.f;
    for (int k = lane; k < nb; k += 32) s += part[(int64_t)b * gx + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[b] = s;
}

// dv += alpha p, r -= alpha A p with alpha = rr / pap; partials of r . r
__global__ void __launch_bounds__(TB) impl_update_kernel(ImplArgs A)
{
    __shared__ float red[TB / 32];
    int b, kb;
    locate(A, b, kb);
    const ClothDesc& D = A.desc[b];
    const int n = D.rows * D.cols;
    const int i = kb * TB + (int)threadIdx.x;
    const float pap = A.pap[b];
    const float alpha = pap > 0.f ? A.rr[b] / pap : 0.f;
    float rr = 0.f;
    if (i < n) {
        const int r = i / D.cols, c = i % D.cols;
        const int64_t o = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int64_t q = o + k * D.plane_stride;
            A.dv[q] = fmaf(alpha, A.p[q], A.dv[q]);
            const float rk = fmaf(-alpha, A.ap[q], A.r[q]);
            A.r[q] = rk;
            rr = fmaf(rk, rk, rr);
        }
    }
    const float s = block_sum(rr, red);
    if (threadIdx.x == 0) A.part[(int64_t)b * A.gx + kb] = s;
}

// p = r + beta p with beta = rr_new / rr; then rr <- rr_new (thread 0 of
// each cloth's first block, after its own use)
__global__ void __launch_bounds__(TB) impl_dir_kernel(ImplArgs A)
{
    int b, kb;
    locate(A, b, kb);
    const ClothDesc& D = A.desc[b];
    const int n = D.rows * D.cols;
    const int i = kb * TB + (int)threadIdx.x;
    if (i >= n) return;
    const float rr = A.rr[b];
    const float beta = rr > 0.f ? A.rr_new[b] / rr : 0.f;
    const int r = i / D.cols, c = i % D.cols;
    const int64_t o = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t q = o + k * D.plane_stride;
        A.p[q] = fmaf(beta, A.p[q], A.r[q]);
    }
}

__global__ void impl_swap_kernel(int B, float* __restrict__ rr, const float* __restrict__ rr_new)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) rr[b] = rr_new[b];
}

// v' = C(v + dv), x' = x + h v', sphere contact, into dst
__global__ void __launch_bounds__(TB) impl_finish_kernel(ImplArgs A, float* __restrict__ dst, int32_t* status)
{
    int b, kb;
    locate(A, b, kb);
    const ClothDesc& D = A.desc[b];
    const int n = D.rows * D.cols;
    const int i = kb * TB + (int)threadIdx.x;
    if (i >= n) return;
    const int r = i / D.cols, c = i % D.cols;
    const int64_t o = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
    const bool pi = pinned_at(D, A.pinmask, r, c);
    float un[3], vn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float v = A.state[o + (3 + k) * D.plane_stride];
        vn[k] = pi ? pin_v(D, k) : v + A.dv[o + k * D.plane_stride];
        un[k] = fmaf(A.h, vn[k], A.state[o + k * D.plane_stride]);
    }
    if (D.sph_on) sphere_contact(D, c, r, D.h, un[0], un[1], un[2], vn[0], vn[1], vn[2]);
    if (!isfinite(un[0] + un[1] + un[2] + vn[0] + vn[1] + vn[2])) atomicOr(status, kStatusNonfinite);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dst[o + k * D.plane_stride] = un[k];
        dst[o + (3 + k) * D.plane_stride] = vn[k];
    }
}

}  // namespace

int implicit_grid_x(int64_t max_nodes) { return (int)((max_nodes + TB - 1) / TB); }
int implicit_block_nodes() { return TB; }

cudaError_t launch_implicit_step(const ClothDesc* desc, const uint32_t* pinmask, int B, int64_t max_nodes,
                                 const int32_t* blk, int n_blocks, const float* state, const float* f_abi, float* dst,
                                 float* vecs, int64_t state_floats, float* part, float* scal, float h, int cg_iters,
                                 int32_t* status, cudaStream_t s)
{
    ImplArgs a{};
    a.desc = desc;
    a.pinmask = pinmask;
    a.state = state;
    a.f_abi = f_abi;
    a.dv = vecs;
    a.r = vecs + state_floats;
    a.p = vecs + 2 * state_floats;
    a.ap = vecs + 3 * state_floats;
    a.part = part;
    a.rr = scal;
    a.rr_new = scal + B;
    a.pap = scal + 2 * B;
    a.blk = blk;
    a.B = B;
    a.gx = implicit_grid_x(max_nodes);
    a.h = h;
    const dim3 grid((unsigned)n_blocks);
    impl_rhs_kernel<<<grid, TB, 0, s>>>(a);
    impl_reduce_kernel<<<B, 32, 0, s>>>(desc, part, a.gx, a.rr);
    for (int it = 0; it < cg_iters; ++it) {
        impl_matvec_kernel<<<grid, TB, 0, s>>>(a);
        impl_reduce_kernel<<<B, 32, 0, s>>>(desc, part, a.gx, a.pap);
        impl_update_kernel<<<grid, TB, 0, s>>>(a);
        impl_reduce_kernel<<<B, 32, 0, s>>>(desc, part, a.gx, a.rr_new);
        impl_dir_kernel<<<grid, TB, 0, s>>>(a);
        impl_swap_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, a.rr, a.rr_new);
    }
    impl_finish_kernel<<<grid, TB, 0, s>>>(a, dst, status);
    return cudaGetLastError();
}

}  // namespace cloth
