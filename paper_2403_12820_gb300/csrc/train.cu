// Training kernels for the Eq. 8 loss (Sec. 3.2.1): the network rollout of
// Fig. 2 on NCHW windows, the loss terms and their seeds, the adjoint of the
// Euler update with pins and of the pressure force, and Adam.
//
// Every kernel works on B windows of H x W nodes, window n being cloth n of
// the context; grid (ceil(H W / 256), B).  Reductions of the loss are
// per-block partial sums, added in a fixed order by one block.
#include "cloth_internal.cuh"
#include "train_internal.cuh"

namespace cloth {
namespace {

constexpr int TB = 256;

__device__ __forceinline__ bool is_free(const ClothDesc& D, const uint32_t* pinmask, int r, int c)
{
    return !((pinmask[D.pin_off + (int64_t)r * D.pin_wpr + (c >> 5)] >> (c & 31)) & 1u);
}

// e = bE (x_E - x_i) - bW (x_W - x_i), n = bN (x_N - x_i) - bS (x_S - x_i)
// from the displacements u of channels 0..2 of z (x = X + u).
struct EN {
    float e[3], n[3];
};
__device__ __forceinline__ EN pressure_vectors(const float* u, int64_t HW, int r, int c, int H, int W, float h)
{
    const int64_t i = (int64_t)r * W + c;
    EN v;
    for (int k = 0; k < 3; ++k) {
        const float ui = u[k * HW + i];
        float e = 0.f, n = 0.f;
        if (c + 1 < W) e += u[k * HW + i + 1] - ui + (k == 0 ? h : 0.f);
        if (c > 0) e -= u[k * HW + i - 1] - ui - (k == 0 ? h : 0.f);
        if (r + 1 < H) n += u[k * HW + i + W] - ui + (k == 1 ? h : 0.f);
        if (r > 0) n -= u[k * HW + i - W] - ui - (k == 1 ? h : 0.f);
        v.e[k] = e;
        v.n[k] = n;
    }
    return v;
}
__device__ __forceinline__ void cross(const float* a, const float* b, float* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Sum of v over the block into part[blockIdx.y * gridDim.x + blockIdx.x].
__device__ void block_sum(float v, float* part)
{
    __shared__ float red[TB / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int k = 0; k < TB / 32; ++k) s += red[k];
        part[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void state_to_z_kernel(const ClothDesc* __restrict__ desc, const float* __restrict__ state,
                                  float* __restrict__ z, int H, int W)
{
    const int n = blockIdx.y;
    const ClothDesc& D = desc[n];
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= HW) return;
    const int r = (int)(i / W), c = (int)(i % W);
    for (int k = 0; k < 6; ++k)
        z[((int64_t)n * 6 + k) * HW + i] = state[D.plane_off + k * D.plane_stride + (int64_t)r * D.pitch + col_pos(c)];
}

// a_true = (f - f_p) / m: the plain step's acceleration without pressure.
__global__ void a_true_kernel(const ClothDesc* __restrict__ desc, const float* __restrict__ f_abi,
                              const float* __restrict__ z, float* __restrict__ a_true, int H, int W)
{
    const int n = blockIdx.y;
    const ClothDesc& D = desc[n];
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= HW) return;
    const int r = (int)(i / W), c = (int)(i % W);
    float fp[3] = {0.f, 0.f, 0.f};
    if (D.p_quarter != 0.f) {
        const EN v = pressure_vectors(z + (int64_t)n * 6 * HW, HW, r, c, H, W, D.h);
        cross(v.e, v.n, fp);
    }
    for (int k = 0; k < 3; ++k)
        a_true[((int64_t)n * 3 + k) * HW + i] = (f_abi[(D.abi_off + i) * 3 + k] - D.p_quarter * fp[k]) * D.inv_m;
}

// Physics target of a network step of stride k (dt_net = k dt): the mean
// acceleration of the k plain steps from the window start, (v_k - v_0) /
// dt_net, less the pressure acceleration at the start (the network step adds
// that itself).  state_k: the packed state after the k plain steps.
__global__ void a_true_stride_kernel(const ClothDesc* __restrict__ desc, const float* __restrict__ state_k,
                                     const float* __restrict__ z, float* __restrict__ a_true, int H, int W)
{
    const int n = blockIdx.y;
    const ClothDesc& D = desc[n];
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= HW) return;
    const int r = (int)(i / W), c = (int)(i % W);
    const float* zi = z + (int64_t)n * 6 * HW;
    float fp[3] = {0.f, 0.f, 0.f};
    if (D.p_quarter != 0.f) {
        const EN v = pressure_vectors(zi, HW, r, c, H, W, D.h);
        cross(v.e, v.n, fp);
    }
    const int64_t o = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
    for (int k = 0; k < 3; ++k) {
        const float vk = state_k[o + (3 + k) * D.plane_stride];
        a_true[((int64_t)n * 3 + k) * HW + i] = (vk - zi[(3 + k) * HW + i]) / D.dt_net - D.p_quarter * fp[k] * D.inv_m;
    }
}

// Fig. 2 update without contact: v' = C(v + dt (a + f_p / m)), u' = u + dt v'.
__global__ void train_euler_kernel(const ClothDesc* __restrict__ desc, const uint32_t* __restrict__ pinmask,
                                   const float* __restrict__ z, const float* __restrict__ a, float* __restrict__ zn,
                                   int H, int W)
{
    const int n = blockIdx.y;
    const ClothDesc& D = desc[n];
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= HW) return;
    const int r = (int)(i / W), c = (int)(i % W);
    const float* zi = z + (int64_t)n * 6 * HW;
    float fp[3] = {0.f, 0.f, 0.f};
    if (D.p_quarter != 0.f) {
        const EN v = pressure_vectors(zi, HW, r, c, H, W, D.h);
        cross(v.e, v.n, fp);
    }
    const bool fr = is_free(D, pinmask, r, c);
    for (int k = 0; k < 3; ++k) {
        const float acc = a[((int64_t)n * 3 + k) * HW + i] + D.p_quarter * fp[k] * D.inv_m;
        const float vn = fr ? fmaf(D.dt_net, acc, zi[(3 + k) * HW + i]) : pin_v(D, k);   // pins move with pin_v
        zn[((int64_t)n * 6 + 3 + k) * HW + i] = vn;
        zn[((int64_t)n * 6 + k) * HW + i] = fmaf(D.dt_net, vn, zi[k * HW + i]);
    }
}

// Data term at one unrolled step: coef_n * sum_free ((X + u - x_target))^2,
// coef_n = (1 - alpha) / (S cnt_n h^2 B).  Optionally adds the seed
// 2 coef_n (X + u - x_target) to gu.
__global__ void data_term_kernel(const ClothDesc* __restrict__ desc, const uint32_t* __restrict__ pinmask,
                                 const float* __restrict__ z, const float* __restrict__ xt,
                                 const float* __restrict__ coef, float* __restrict__ gu, float* __restrict__ part,
                                 int H, int W)
{
    const int n = blockIdx.y;
    const ClothDesc& D = desc[n];
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    float acc = 0.f;
    if (i < HW) {
        const int r = (int)(i / W), c = (int)(i % W);
        if (is_free(D, pinmask, r, c)) {
            const double X[3] = {(double)c * D.h, (double)r * D.h, 0.0};
            for (int k = 0; k < 3; ++k) {
                // x_target - X in FP64, so the difference keeps its digits
                const float tgt_u = (float)((double)xt[(D.abi_off + i) * 3 + k] - X[k]);
                const float d = z[((int64_t)n * 6 + k) * HW + i] - tgt_u;
                acc = fmaf(coef[n] * d, d, acc);
                if (gu) gu[((int64_t)n * 3 + k) * HW + i] += 2.f * coef[n] * d;
            }
        }
    }
    if (part) block_sum(acc, part);
}

// Physics term: coef_n * sum_free (a0 - a_true)^2, coef_n = alpha / (cnt_n
// g^2 B); seed ga0 = 2 coef_n (a0 - a_true) on free nodes.
__global__ void phys_term_kernel(const ClothDesc* __restrict__ desc, const uint32_t* __restrict__ pinmask,
                                 const float* __restrict__ a0, const float* __restrict__ at,
                                 const float* __restrict__ coef, float* __restrict__ ga0, float* __restrict__ part,
                                 int H, int W)
{
    const int n = blockIdx.y;
    const ClothDesc& D = desc[n];
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    float acc = 0.f;
    if (i < HW) {
        const int r = (int)(i / W), c = (int)(i % W);
        const bool fr = is_free(D, pinmask, r, c);
        for (int k = 0; k < 3; ++k) {
            const int64_t j = ((int64_t)n * 3 + k) * HW + i;
            const float d = a0[j] - at[j];
            if (fr) acc = fmaf(coef[n] * d, d, acc);
            ga0[j] = fr ? 2.f * coef[n] * d : 0.f;
        }
    }
    block_sum(acc, part);
}

__global__ void sum_partials_kernel(const float* __restrict__ part, int count, float* __restrict__ out)
{
    __shared__ float red[TB];
    float s = 0.f;
    for (int k = threadIdx.x; k < count; k += TB) s += part[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = TB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Adjoint of x_t = x_{t-1} + dt v_t, v_t = C(v_{t-1} + dt (a + f_p / m)):
// gv += dt gu; w = free gv; ga = dt w (+ ga0); gfp = dt w / m; gv <- w.
__global__ void euler_adjoint_kernel(const ClothDesc* __restrict__ desc, const uint32_t* __restrict__ pinmask,
                                     const float* __restrict__ gu, float* __restrict__ gv,
                                     const float* __restrict__ ga0, float* __restrict__ ga, float* __restrict__ gfp,
                                     int H, int W)
{
    const int n = blockIdx.y;
    const ClothDesc& D = desc[n];
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= HW) return;
    const int r = (int)(i / W), c = (int)(i % W);
    const bool fr = is_free(D, pinmask, r, c);
    for (int k = 0; k < 3; ++k) {
        const int64_t j = ((int64_t)n * 3 + k) * HW + i;
        const float w = fr ? fmaf(D.dt_net, gu[j], gv[j]) : 0.f;
        gv[j] = w;
        ga[j] = D.dt_net * w + (ga0 ? ga0[j] : 0.f);
        gfp[j] = D.dt_net * w * D.inv_m;
    }
}

// Pressure adjoint, pass 1: with f_p = (p/4) e x n and G = (p/4) gfp,
// ge = n x G and gn = G x e at every node.
__global__ void pvjp1_kernel(const ClothDesc* __restrict__ desc, const float* __restrict__ z,
                             const float* __restrict__ gfp, float* __restrict__ ge, float* __restrict__ gn, int H,
                             int W)
{
    const int n = blockIdx.y;
    const ClothDesc& D = desc[n];
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= HW) return;
    const int r = (int)(i / W), c = (int)(i % W);
    const EN v = pressure_vectors(z + (int64_t)n * 6 * HW, HW, r, c, H, W, D.h);
    float G[3], a[3], b[3];
    for (int k = 0; k < 3; ++k) G[k] = D.p_quarter * gfp[((int64_t)n * 3 + k) * HW + i];
    cross(v.n, G, a);
    cross(G, v.e, b);
    for (int k = 0; k < 3; ++k) {
        ge[((int64_t)n * 3 + k) * HW + i] = a[k];
        gn[((int64_t)n * 3 + k) * HW + i] = b[k];
    }
}

// Pass 2, gathered per node j (e, n depend on x_j and its 4 neighbours):
// gx_j += (bW - bE) ge_j + (bS - bN) gn_j + bW ge_W(j) - bE ge_E(j)
//       + bS gn_S(j) - bN gn_N(j).
__global__ void pvjp2_kernel(const float* __restrict__ ge, const float* __restrict__ gn, float* __restrict__ gu,
                             int H, int W)
{
    const int n = blockIdx.y;
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= HW) return;
    const int r = (int)(i / W), c = (int)(i % W);
    const bool bE = c + 1 < W, bW = c > 0, bN = r + 1 < H, bS = r > 0;
    for (int k = 0; k < 3; ++k) {
        const float* e = ge + ((int64_t)n * 3 + k) * HW;
        const float* g = gn + ((int64_t)n * 3 + k) * HW;
        float s = ((bW ? 1.f : 0.f) - (bE ? 1.f : 0.f)) * e[i] + ((bS ? 1.f : 0.f) - (bN ? 1.f : 0.f)) * g[i];
        if (bW) s += e[i - 1];
        if (bE) s -= e[i + 1];
        if (bS) s += g[i - W];
        if (bN) s -= g[i + W];
        gu[((int64_t)n * 3 + k) * HW + i] += s;
    }
}

// gu += dL/du, gv += dL/dv from the cell's input gradient gz [B][6][H][W].
__global__ void add_gz_kernel(const float* __restrict__ gz, float* __restrict__ gu, float* __restrict__ gv, int H,
                              int W)
{
    const int n = blockIdx.y;
    const int64_t HW = (int64_t)H * W, i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= HW) return;
    for (int k = 0; k < 3; ++k) {
        gu[((int64_t)n * 3 + k) * HW + i] += gz[((int64_t)n * 6 + k) * HW + i];
        gv[((int64_t)n * 3 + k) * HW + i] += gz[((int64_t)n * 6 + 3 + k) * HW + i];
    }
}

// Entries whose mask byte is 0 (mask set) keep w, m and v: frozen groups.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, const uint8_t* __restrict__ mask, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (mask && !mask[i])) return;
    const float mi = fmaf(b1, m[i], (1.f - b1) * g[i]);
    const float vi = fmaf(b2, v[i], (1.f - b2) * g[i] * g[i]);
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

dim3 grid2(int H, int W, int B) { return dim3((unsigned)(((int64_t)H * W + TB - 1) / TB), (unsigned)B); }

}  // namespace

int train_blocks(int H, int W, int B) { const dim3 g = grid2(H, W, B); return (int)(g.x * g.y); }

cudaError_t launch_state_to_z(const ClothDesc* d, const float* state, float* z, int B, int H, int W, cudaStream_t s)
{
    state_to_z_kernel<<<grid2(H, W, B), TB, 0, s>>>(d, state, z, H, W);
    return cudaGetLastError();
}
cudaError_t launch_a_true_stride(const ClothDesc* d, const float* state_k, const float* z, float* at, int B, int H,
                                 int W, cudaStream_t s)
{
    a_true_stride_kernel<<<grid2(H, W, B), TB, 0, s>>>(d, state_k, z, at, H, W);
    return cudaGetLastError();
}
cudaError_t launch_a_true(const ClothDesc* d, const float* f_abi, const float* z, float* at, int B, int H, int W,
                          cudaStream_t s)
{
    a_true_kernel<<<grid2(H, W, B), TB, 0, s>>>(d, f_abi, z, at, H, W);
    return cudaGetLastError();
}
cudaError_t launch_train_euler(const ClothDesc* d, const uint32_t* pins, const float* z, const float* a, float* zn,
                               int B, int H, int W, cudaStream_t s)
{
    train_euler_kernel<<<grid2(H, W, B), TB, 0, s>>>(d, pins, z, a, zn, H, W);
    return cudaGetLastError();
}
cudaError_t launch_data_term(const ClothDesc* d, const uint32_t* pins, const float* z, const float* xt,
                             const float* coef, float* gu, float* part, int B, int H, int W, cudaStream_t s)
{
    data_term_kernel<<<grid2(H, W, B), TB, 0, s>>>(d, pins, z, xt, coef, gu, part, H, W);
    return cudaGetLastError();
}
cudaError_t launch_phys_term(const ClothDesc* d, const uint32_t* pins, const float* a0, const float* at,
                             const float* coef, float* ga0, float* part, int B, int H, int W, cudaStream_t s)
{
    phys_term_kernel<<<grid2(H, W, B), TB, 0, s>>>(d, pins, a0, at, coef, ga0, part, H, W);
    return cudaGetLastError();
}
cudaError_t launch_sum_partials(const float* part, int count, float* out, cudaStream_t s)
{
    sum_partials_kernel<<<1, TB, 0, s>>>(part, count, out);
    return cudaGetLastError();
}
cudaError_t launch_euler_adjoint(const ClothDesc* d, const uint32_t* pins, const float* gu, float* gv,
                                 const float* ga0, float* ga, float* gfp, int B, int H, int W, cudaStream_t s)
{
    euler_adjoint_kernel<<<grid2(H, W, B), TB, 0, s>>>(d, pins, gu, gv, ga0, ga, gfp, H, W);
    return cudaGetLastError();
}
cudaError_t launch_pressure_vjp(const ClothDesc* d, const float* z, const float* gfp, float* ge, float* gn, float* gu,
                                int B, int H, int W, cudaStream_t s)
{
    pvjp1_kernel<<<grid2(H, W, B), TB, 0, s>>>(d, z, gfp, ge, gn, H, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    pvjp2_kernel<<<grid2(H, W, B), TB, 0, s>>>(ge, gn, gu, H, W);
    return cudaGetLastError();
}
cudaError_t launch_add_gz(const float* gz, float* gu, float* gv, int B, int H, int W, cudaStream_t s)
{
    add_gz_kernel<<<grid2(H, W, B), TB, 0, s>>>(gz, gu, gv, H, W);
    return cudaGetLastError();
}
cudaError_t launch_adam(float* w, const float* g, float* m, float* v, const uint8_t* mask, int n, int t, float lr,
                        float b1, float b2, float eps, cudaStream_t s)
{
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(w, g, m, v, mask, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace cloth
