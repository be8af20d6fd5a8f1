// The trunk's second 3x3 convolution, 32 channels to 32 (Eq. 6: phi =
// W2 (*) phi1, xi = W2 (*) xi1), and its adjoint with respect to the input
// (the transposed convolution of the backward pass), on the tcgen05 tensor
// cores at FP32 precision: every FP32 operand x is held as two BF16 parts,
// x = hi + lo with hi = BF16(x) and lo = BF16(x - hi), and each product as
// three BF16 MMAs into an FP32 accumulator (hi hi + hi lo + lo hi; the
// dropped lo lo term is at most 2^-18 of the product).
//
// Implicit GEMM per image tile: the tile's input region (its R output rows
// plus a 1-node halo, at a pitch of CP nodes per row) is staged channel-last
// as BF16, node j of channel group g (channels 8 g .. 8 g + 7) at row
// g * N0BUF + j of the operand, so a 3 x 3 tap (ky, kx) is the operand
// shifted by ky * CP + kx rows (a descriptor offset); M = 128 consecutive
// output-region nodes ("a chunk"), N = 32 output channels, K = 16 = two
// channel groups: per chunk 9 taps x 2 K halves x 3 parts = 54 MMAs.  The
// output region's junk nodes (the 2 halo columns of each row and the tail
// of the last chunk) are computed and dropped.  Two CTAs of 4 warps per SM
// (one stages and reads back while the other's MMAs run); every wait on the
// tensor cores is bounded, a timeout sets the status bit and the CTA stops.
#include <cuda_bf16.h>

#include "net_internal.cuh"
#include "tc_ptx.cuh"

namespace cloth {
namespace {

constexpr int NTC = 128;                   // threads per CTA: warp w reads TMEM lanes [32 w, +32)
constexpr uint32_t kConvWait = 1u << 24;   // polls of a bounded wait

// Tile shape: CP nodes per region row (CP - 2 output columns), R output rows,
// C chunks of 128 output-region nodes.
template <int CPV, int RV>
struct ConvShape {
    static constexpr int CP = CPV, R = RV, WO = CP - 2;
    static constexpr int C = (R * CP + 127) / 128;
    static constexpr int N0 = (R + 2) * CP;                                  // input-region nodes
    static constexpr int N0BUF = (C * 128 + 2 * CP + 2 + 15) / 16 * 16;      // rows the MMAs read
    static constexpr int kAPart = 4 * N0BUF * 16;                            // bytes of one part of A
    static constexpr int kBPart = 9 * 4 * 32 * 16;                           // [tap][group][o 32][8] bf16
    static constexpr int oA = 0, oB = 2 * kAPart, oBar = oB + 2 * kBPart, oSlot = oBar + 16;
    static constexpr int kSmem = oSlot + 16;
    static constexpr uint32_t kCols = C * 32 <= 32 ? 32 : (C * 32 <= 64 ? 64 : (C * 32 <= 128 ? 128 : 256));
    static_assert(N0BUF >= N0 && kSmem <= 113 * 1024, "two CTAs per SM");
};
using Narrow = ConvShape<32, 12>;   // images up to 30 wide: 12 x 30 output tiles, 3 chunks
using Wide = ConvShape<66, 5>;      // wider images: 5 x 64 output tiles, 3 chunks

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&b);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// out[img][o][y][x] = sum_{i, ky, kx} Wt(o, i, ky, kx) in[img][i][y+ky-1][x+kx-1],
// zero outside the image; NCHW with an image stride of 32 H W floats.
// Wt(o, i, tap) = W2[o][i][tap], or W2[i][o][8 - tap] for the adjoint.
template <class S, bool TRANSPOSED>
__global__ void __launch_bounds__(NTC, 2)
    conv32_tc_kernel(const float* __restrict__ in, float* __restrict__ out, const float* __restrict__ w, int images,
                     int H, int W, int32_t* __restrict__ status)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = tc::smem_u32(sm);
    const uint32_t bar = sbase + S::oBar, bar_drain = sbase + S::oBar + 8;
    volatile uint32_t* sTmem = reinterpret_cast<uint32_t*>(sm + S::oSlot);
    const int64_t HW = (int64_t)H * W;
    const int tiles_x = (W + S::WO - 1) / S::WO, tiles_y = (H + S::R - 1) / S::R;
    const int n_tiles = images * tiles_y * tiles_x;

    // B: both parts of the 9 x 32 x 32 weights, [part][tap][group][o][8]
    for (int e = tid; e < 9 * 32 * 32; e += NTC) {
        const int tap = e / 1024, o = (e / 32) % 32, i = e % 32;
        const float v = TRANSPOSED ? w[kOffW2 + (i * kC + o) * 9 + (8 - tap)] : w[kOffW2 + (o * kC + i) * 9 + tap];
        const float hi = bf16r(v);
        const int r = ((tap * 4 + i / 8) * 32 + o) * 8 + i % 8;
        reinterpret_cast<__nv_bfloat16*>(sm + S::oB)[r] = __float2bfloat16_rn(hi);
        reinterpret_cast<__nv_bfloat16*>(sm + S::oB + S::kBPart)[r] = __float2bfloat16_rn(v - hi);
    }
    // A rows N0 .. N0BUF are read only by junk output nodes; keep them zero
    for (int e = tid; e < 2 * 4 * (S::N0BUF - S::N0); e += NTC) {
        const int pg = e / (S::N0BUF - S::N0);
        reinterpret_cast<uint4*>(sm + S::oA)[pg * S::N0BUF + S::N0 + e % (S::N0BUF - S::N0)] = make_uint4(0, 0, 0, 0);
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(bar_drain, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(sbase + S::oSlot, S::kCols);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *sTmem;
    uint32_t phase = 0;
    bool timed_out = false;

    // descriptors: A [group][node][8] (K-adjacent core matrices N0BUF rows
    // apart, 8-node groups 128 bytes apart); B [group][o][8] per tap
    const uint64_t dA = tc::sdesc(sbase + S::oA, S::N0BUF * 16, 128);
    const uint64_t dB = tc::sdesc(sbase + S::oB, 32 * 16, 128);
    constexpr uint64_t kALo = S::kAPart >> 4, kBLo = S::kBPart >> 4;

    for (int tile = blockIdx.x; tile < n_tiles && !timed_out; tile += gridDim.x) {
        const int img = tile / (tiles_y * tiles_x), r = tile % (tiles_y * tiles_x);
        const int y0 = (r / tiles_x) * S::R, x0 = (r % tiles_x) * S::WO;
        const float* src = in + (int64_t)img * kC * HW;
        // 1. the input region, channel-last, both parts: one node and one
        // channel group (8 loads, one 16-byte store per part) per item, the
        // loads of kItems items in flight before any is stored
        constexpr int kItems = 4;
        for (int it0 = tid; it0 < 4 * S::N0; it0 += kItems * NTC) {
            float v[kItems][8];
#pragma unroll
            for (int q = 0; q < kItems; ++q) {
                const int it = it0 + q * NTC, g = it / S::N0, j = it % S::N0;
                const int y = y0 - 1 + j / S::CP, x = x0 - 1 + j % S::CP;
                const bool inside = it < 4 * S::N0 && y >= 0 && y < H && x >= 0 && x < W;
#pragma unroll
                for (int e = 0; e < 8; ++e) v[q][e] = inside ? __ldg(src + (8 * g + e) * HW + (int64_t)y * W + x) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < kItems; ++q) {
                const int it = it0 + q * NTC;
                if (it >= 4 * S::N0) break;
                float h[8], l[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    h[e] = bf16r(v[q][e]);
                    l[e] = v[q][e] - h[e];
                }
                uint4* a = reinterpret_cast<uint4*>(sm + S::oA) + (it / S::N0) * S::N0BUF + it % S::N0;
                a[0] = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
                a[4 * S::N0BUF] = make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // 2. one thread issues every chunk's MMAs
        if (tid == 0) {
            for (int c = 0; c < S::C; ++c) {
                const uint32_t d = tmem + 32u * (uint32_t)c;
                bool acc = false;
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const uint64_t off = (uint64_t)(c * 128 + (tap / 3) * S::CP + tap % 3);
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh) {
                        const uint64_t a = dA + (uint64_t)(2 * kh * S::N0BUF) + off;
                        const uint64_t b = dB + (uint64_t)((tap * 4 + 2 * kh) * 32);
                        tc::mma_bf16(d, a, b, tc::idesc_bf16(128, 32), acc);
                        tc::mma_bf16(d, a, b + kBLo, tc::idesc_bf16(128, 32), true);
                        tc::mma_bf16(d, a + kALo, b, tc::idesc_bf16(128, 32), true);
                        acc = true;
                    }
                }
            }
            tc::mma_commit(bar);
        }
        // 3. read back: warp w takes TMEM lanes [32 w, +32) of every chunk
        const bool ok = tc::mbar_wait(bar, phase, kConvWait);
        phase ^= 1u;
        tc::fence_after();
        if (ok) {
            for (int c = 0; c < S::C; ++c) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32u * (uint32_t)c, v);
                tc::tmem_wait_ld();
                const int j = c * 128 + 32 * warp + lane, ry = j / S::CP, rx = j % S::CP;
                const int y = y0 + ry, x = x0 + rx;
                if (ry < S::R && rx < S::WO && y < H && x < W) {
                    float* o = out + (int64_t)img * kC * HW + (int64_t)y * W + x;
#pragma unroll
                    for (int k = 0; k < 32; ++k) o[k * HW] = v[k];
                }
            }
        }
        tc::fence_before();
        if (__syncthreads_or(!ok)) timed_out = true;   // the next tile rewrites A
    }

    // tear-down: the MMAs issued are done (bounded) before tensor memory is freed
    if (timed_out && tid == 0 && status) atomicOr(status, kStatusTimeout);
    if (tid == 0) tc::mma_commit(bar_drain);
    __syncthreads();
    if (warp == 0) {
        if (!tc::mbar_wait(bar_drain, 0, kConvWait) && lane == 0 && status) atomicOr(status, kStatusTimeout);
        tc::fence_after();
        tc::tmem_dealloc(tmem, S::kCols);
    }
}

template <class S, bool T>
cudaError_t launch_shape(const float* in, float* out, const float* w, int images, int H, int W, int sm_count,
                         int32_t* status, cudaStream_t s)
{
    const int n_tiles = images * ((H + S::R - 1) / S::R) * ((W + S::WO - 1) / S::WO);
    const int grid = n_tiles < 2 * sm_count ? n_tiles : 2 * sm_count;
    conv32_tc_kernel<S, T><<<grid, NTC, S::kSmem, s>>>(in, out, w, images, H, W, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t conv32_tc_init()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern, int bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set(conv32_tc_kernel<Narrow, false>, Narrow::kSmem);
    set(conv32_tc_kernel<Narrow, true>, Narrow::kSmem);
    set(conv32_tc_kernel<Wide, false>, Wide::kSmem);
    set(conv32_tc_kernel<Wide, true>, Wide::kSmem);
    return e;
}

cudaError_t launch_conv32_tc(const float* in, float* out, const float* w, bool transposed, int images, int H, int W,
                             int32_t* status, cudaStream_t s)
{
    if (images <= 0 || H <= 0 || W <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (W <= Narrow::WO)
        return transposed ? launch_shape<Narrow, true>(in, out, w, images, H, W, sms, status, s)
                          : launch_shape<Narrow, false>(in, out, w, images, H, W, sms, status, s);
    return transposed ? launch_shape<Wide, true>(in, out, w, images, H, W, sms, status, s)
                      : launch_shape<Wide, false>(in, out, w, images, H, W, sms, status, s);
}

}  // namespace cloth
