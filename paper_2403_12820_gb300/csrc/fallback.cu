// Plain-step fallback of the network rollout: the framework of Fig. 2 can
// couple the network with the physics-based simulator, which here serves
// as the judge of the network step.  On a check step both steps start from
// the same state; a cloth whose largest node-position difference exceeds
// the bound is switched to the plain step for the rest of the rollout.
#include <cfloat>

#include "cloth_internal.cuh"

namespace cloth {
namespace {

constexpr int TB = 256;

// resid[b] = max over the nodes of cloth b (still in network mode) of
// |u_net - u_plain|, +inf where that difference is not finite; positive
// floats (+inf included) order like their bit patterns.
__global__ void residual_kernel(const ClothDesc* __restrict__ desc, const int32_t* __restrict__ mode,
                                const float* __restrict__ net, const float* __restrict__ plain,
                                float* __restrict__ resid)
{
    const int b = blockIdx.y;
    if (mode[b] != kModeNet) return;
    const ClothDesc& D = desc[b];
    const int64_t n = (int64_t)D.rows * D.cols;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        const int r = (int)(i / D.cols), c = (int)(i % D.cols);
        const int64_t o = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
        float d2 = 0.f;
        for (int k = 0; k < 3; ++k) {
            const float d = net[o + k * D.plane_stride] - plain[o + k * D.plane_stride];
            d2 = fmaf(d, d, d2);
        }
        // a non-finite difference (a network result gone NaN or infinite)
        // counts as an infinite residual: fmaxf would drop a NaN
        m = fmaxf(m, d2 <= FLT_MAX ? sqrtf(d2) : __int_as_float(0x7f800000));
    }
    for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, s));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(resid + b), __float_as_int(m));
}

// Cloths that stay in network mode take the network result; the others keep
// the plain result already in dst.
__global__ void merge_kernel(const ClothDesc* __restrict__ desc, const int32_t* __restrict__ mode,
                             const float* __restrict__ resid, float bound, const float* __restrict__ net,
                             float* __restrict__ dst)
{
    const int b = blockIdx.y;
    if (mode[b] != kModeNet || !(resid[b] <= bound)) return;
    const ClothDesc& D = desc[b];
    const int64_t n = (int64_t)D.rows * D.cols;
    for (int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        const int r = (int)(i / D.cols), c = (int)(i % D.cols);
        const int64_t o = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
        for (int k = 0; k < 6; ++k) dst[o + k * D.plane_stride] = net[o + k * D.plane_stride];
    }
}

__global__ void latch_kernel(int B, int32_t* __restrict__ mode, const float* __restrict__ resid, float bound,
                             float* __restrict__ last)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (mode[b] != kModeNet) return;   // keeps the residual that switched it
    if (!(resid[b] <= bound)) mode[b] = kModePlain;
    last[b] = resid[b];
}

}  // namespace

cudaError_t launch_fallback_check(const ClothDesc* desc, int B, int64_t max_nodes, int32_t* mode, float* resid,
                                  float* last, float bound, const float* net, float* dst, cudaStream_t s)
{
    const dim3 grid((unsigned)((max_nodes + TB - 1) / TB < 1024 ? (max_nodes + TB - 1) / TB : 1024), (unsigned)B);
    cudaError_t e = cudaMemsetAsync(resid, 0, sizeof(float) * B, s);
    if (e != cudaSuccess) return e;
    residual_kernel<<<grid, TB, 0, s>>>(desc, mode, net, dst, resid);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    merge_kernel<<<grid, TB, 0, s>>>(desc, mode, resid, bound, net, dst);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    latch_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, mode, resid, bound, last);
    return cudaGetLastError();
}

}  // namespace cloth
