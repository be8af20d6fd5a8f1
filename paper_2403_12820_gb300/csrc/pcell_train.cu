// The literal cell (Sec. 3.2, Eq. 6-7, Fig. 1) on the training layout: B
// windows of H x W nodes, z [B][6][H][W] = (u_x, u_y, u_z, v_x, v_y, v_z)
// with u = x - X, as the Eq. 8 unroll keeps them.  Forward a [B][3][H][W];
// backward: the gradient with respect to z (written) and to the 39 trainable
// parameters (added to grad_w; alpha is a fixed hyper-parameter).
//
// Grid (ceil(H W / 256), B), one thread per node.  The backward gathers:
// node i gets -dt/dphi of each of its own channels and +dt/dphi of the
// channel of each neighbour j that points back at i (phi_j = -phi_i,
// xi_j = -xi_i), so no atomics are needed.  The weight gradient is summed
// per block and the block partials are added in a fixed order: the result is
// bitwise reproducible.
#include "cloth_internal.cuh"
#include "train_internal.cuh"

namespace cloth {
namespace {

constexpr int TB = 256;
constexpr int kW = 40;    // w_L[12], w_N[12], w_D[12], b_L[3], alpha
constexpr int kG = 39;    // trainable entries

// channel offsets (row, column): E W N S NE NW SE SW E2 W2 N2 S2, and the
// channel of the neighbour that points back
__host__ __device__ constexpr int ch_dy(int c)
{
    return c == 2 || c == 4 || c == 5 ? 1 : (c == 3 || c == 6 || c == 7 ? -1 : (c == 10 ? 2 : (c == 11 ? -2 : 0)));
}
__host__ __device__ constexpr int ch_dx(int c)
{
    return c == 0 || c == 4 || c == 6 ? 1 : (c == 1 || c == 5 || c == 7 ? -1 : (c == 8 ? 2 : (c == 9 ? -2 : 0)));
}
__host__ __device__ constexpr int ch_opp(int c)
{
    return c == 0 ? 1 : c == 1 ? 0 : c == 2 ? 3 : c == 3 ? 2 : c == 4 ? 7 : c == 7 ? 4 : c == 5 ? 6 : c == 6 ? 5
         : c == 8 ? 9 : c == 9 ? 8 : c == 10 ? 11 : 10;
}

__global__ void __launch_bounds__(TB) pcell_fwd_z_kernel(const ClothDesc* __restrict__ desc,
                                                        const float* __restrict__ w, const float* __restrict__ z,
                                                        float* __restrict__ a, int H, int W)
{
    __shared__ float sw[kW];
    if (threadIdx.x < kW) sw[threadIdx.x] = w[threadIdx.x];
    __syncthreads();
    const int n = blockIdx.y;
    const int64_t HW = (int64_t)H * W;
    const int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= HW) return;
    const int r = (int)(i / W), c = (int)(i % W);
    const float h = desc[n].h, alpha = sw[39];
    const float* zn = z + (int64_t)n * 6 * HW;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float acc = sw[36 + k];
        const float ui = zn[k * HW + i], vi = zn[(3 + k) * HW + i];
#pragma unroll
        for (int ch = 0; ch < 12; ++ch) {
            const int dy = ch_dy(ch), dx = ch_dx(ch);
            if (r + dy < 0 || r + dy >= H || c + dx < 0 || c + dx >= W) continue;
            const int64_t j = i + (int64_t)dy * W + dx;
            const float lat = k == 0 ? (float)dx * h : (k == 1 ? (float)dy * h : 0.f);
            const float phi = lat + (zn[k * HW + j] - ui);
            const float xi = zn[(3 + k) * HW + j] - vi;
            const float s = phi * rsqrt_ftz(fmaf(alpha * phi, phi, 1.f));   // the argument is >= 1
            acc = fmaf(sw[ch], phi, fmaf(s, fmaf(sw[24 + ch], xi, sw[12 + ch]), acc));
        }
        a[((int64_t)n * 3 + k) * HW + i] = acc;
    }
}

__global__ void __launch_bounds__(TB) pcell_bwd_z_kernel(const ClothDesc* __restrict__ desc,
                                                        const float* __restrict__ w, const float* __restrict__ z,
                                                        const float* __restrict__ ga, float* __restrict__ gz,
                                                        float* __restrict__ part, int H, int W)
{
    __shared__ float sw[kW];
    __shared__ float red[TB / 32][kW];
    if (threadIdx.x < kW) sw[threadIdx.x] = w[threadIdx.x];
    __syncthreads();
    const int n = blockIdx.y;
    const int64_t HW = (int64_t)H * W;
    const int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    float gw[kG];
#pragma unroll
    for (int p = 0; p < kG; ++p) gw[p] = 0.f;
    if (i < HW) {
        const int r = (int)(i / W), c = (int)(i % W);
        const float h = desc[n].h, alpha = sw[39];
        const float* zn = z + (int64_t)n * 6 * HW;
        const float* gan = ga + (int64_t)n * 3 * HW;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float gi = gan[k * HW + i];
            const float ui = zn[k * HW + i], vi = zn[(3 + k) * HW + i];
            gw[36 + k] += gi;
            float gu = 0.f, gv = 0.f;
#pragma unroll
            for (int ch = 0; ch < 12; ++ch) {
                const int dy = ch_dy(ch), dx = ch_dx(ch), op = ch_opp(ch);
                if (r + dy < 0 || r + dy >= H || c + dx < 0 || c + dx >= W) continue;
                const int64_t j = i + (int64_t)dy * W + dx;
                const float lat = k == 0 ? (float)dx * h : (k == 1 ? (float)dy * h : 0.f);
                const float phi = lat + (zn[k * HW + j] - ui);
                const float xi = zn[(3 + k) * HW + j] - vi;
                const float rq = rsqrt_ftz(fmaf(alpha * phi, phi, 1.f));   // the argument is >= 1
                const float s = phi * rq, ds = rq * rq * rq;
                gw[ch] = fmaf(gi, phi, gw[ch]);
                gw[12 + ch] = fmaf(gi, s, gw[12 + ch]);
                gw[24 + ch] = fmaf(gi * xi, s, gw[24 + ch]);
                // node i's own channel ch ...
                gu -= gi * fmaf(fmaf(sw[24 + ch], xi, sw[12 + ch]), ds, sw[ch]);
                gv -= gi * sw[24 + ch] * s;
                // ... and neighbour j's channel op, which sees -phi, -xi
                const float gj = gan[k * HW + j];
                gu += gj * fmaf(fmaf(-sw[24 + op], xi, sw[12 + op]), ds, sw[op]);
                gv -= gj * sw[24 + op] * s;
            }
            gz[((int64_t)n * 6 + k) * HW + i] = gu;
            gz[((int64_t)n * 6 + 3 + k) * HW + i] = gv;
        }
    }
    // block sums of the parameter gradient, in a fixed order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < kG; ++p) {
        float v = gw[p];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][p] = v;
    }
    __syncthreads();
    if (threadIdx.x < kG) {
        float s = 0.f;
        for (int q = 0; q < TB / 32; ++q) s += red[q][threadIdx.x];
        part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kW + threadIdx.x] = s;
    }
}

// grad_w[p] += sum over blocks of part[block][p], blocks in order (p < 39)
__global__ void pcell_wgrad_reduce_kernel(const float* __restrict__ part, int blocks, float* __restrict__ gw)
{
    const int p = threadIdx.x;
    if (p >= kG) return;
    float s = 0.f;
    for (int b = 0; b < blocks; ++b) s += part[(int64_t)b * kW + p];
    gw[p] += s;
}

dim3 grid2(int H, int W, int B) { return dim3((unsigned)(((int64_t)H * W + TB - 1) / TB), (unsigned)B); }

}  // namespace

int pcell_train_blocks(int H, int W, int B) { const dim3 g = grid2(H, W, B); return (int)(g.x * g.y); }

cudaError_t launch_pcell_fwd_z(const ClothDesc* d, const float* w, const float* z, float* a, int B, int H, int W,
                               cudaStream_t s)
{
    pcell_fwd_z_kernel<<<grid2(H, W, B), TB, 0, s>>>(d, w, z, a, H, W);
    return cudaGetLastError();
}

cudaError_t launch_pcell_bwd_z(const ClothDesc* d, const float* w, const float* z, const float* ga, float* gz,
                               float* part, float* grad_w, int B, int H, int W, cudaStream_t s)
{
    const dim3 g = grid2(H, W, B);
    pcell_bwd_z_kernel<<<g, TB, 0, s>>>(d, w, z, ga, gz, part, H, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    pcell_wgrad_reduce_kernel<<<1, 64, 0, s>>>(part, (int)(g.x * g.y), grad_w);
    return cudaGetLastError();
}

}  // namespace cloth
