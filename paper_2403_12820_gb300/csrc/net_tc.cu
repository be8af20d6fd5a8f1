// The CNN cell (Sec. 3.2, Eq. 6-7) and the network step (Fig. 2) fused
// into one kernel on the tcgen05 tensor cores: BF16 operands in shared
// memory, FP32 accumulators in tensor memory.
//
// One CTA (4 warps) per SM loops over tiles of R x WO output nodes.  With
// the layer pitch PT = WO + 4, node (ry, rx) of a layer region has the
// linear index ry * PT + rx, and an M = 128 MMA covers 128 consecutive
// linear indices ("a chunk").  Per tile:
//   1. stage u, v of the (R+6) x (WO+6) input tile (3-node halo) in smem;
//   2. layer 1 (Eq. 6): per chunk of the (R+4) x PT layer-1 region, an
//      im2col A tile (K = 3 channels x 9 taps = 27, padded to 32) per field,
//      two MMAs per field against W1[:, field] -> phi1, xi1 (BF16, zero
//      outside the cloth) in smem, K-major core-matrix layout;
//   3. layer 2 as implicit GEMM: for each chunk of the (R+2)-row layer-2
//      region and each tap (dy, dx), the A operand is the layer-1 buffer
//      shifted by dy * PT + dx rows — a descriptor offset, no copy.  The
//      position field multiplies by [P.W2 | WL_tap.W2] (N = 64): it yields
//      t = P phi (the pre-activation of s) and the 27 partial sums
//      q_tap,co = sum_c WL[co][c][tap] phi_c directly, since phi enters
//      Eq. 7 only linearly through P and WL; the velocity field multiplies
//      by W2 (N = 32) -> xi;
//   4. epilogue per layer-2 node: s = tanh(t), N + D = WN s + WD (xi . s),
//      q kept in smem (zero outside the cloth: WL's zero padding);
//   5. per output node: L = bL + sum_tap q_tap at the tap's neighbour,
//      a = out_scale (L + N + D); then (step mode) v <- C(v + dt (a + f_p /
//      m)), u <- u + dt v, sphere contact, store.
// Every wait on the tensor cores is bounded; a timeout sets a status bit
// and the kernel returns after releasing its tensor memory.
#include <cuda_bf16.h>

#include "net_internal.cuh"
#include "tc_ptx.cuh"

namespace cloth {
namespace {

constexpr int R = 12, WO = 28, PT = WO + 4;   // output rows, output columns, layer pitch
constexpr int IH = R + 6, IW = WO + 6;          // input tile (3-node halo)
constexpr int N1 = (R + 4) * PT;                // layer-1 nodes of a tile
constexpr int N2 = (R + 2) * PT;                // layer-2 positions (pitch PT)
constexpr int C1 = N1 / 128;                    // layer-1 chunks
constexpr int C2 = (N2 + 127) / 128;            // layer-2 chunks
constexpr int N1BUF = (C2 * 128 + 2 * PT + 2 + 127) / 128 * 128;   // + rows read by shifted taps
constexpr int NTH = 256;                         // 8 warps; warps w and w + 4 share TMEM lanes
constexpr uint32_t kWaitLimit = 1u << 24;
static_assert(N1 % 128 == 0, "layer-1 region must be whole chunks");
static_assert(N1BUF >= N1, "layer-1 buffer");

// packed BF16 weights: B1 [field][plane][32][8], B2p [tap][plane][64][8],
// B2x [tap][plane][32][8]; plane = 8 consecutive K (input) channels
constexpr int kB1 = 2 * 4 * 32 * 16, kB2p = 9 * 4 * 64 * 16, kB2x = 9 * 4 * 32 * 16;
constexpr int kPack = kB1 + kB2p + kB2x;

// shared memory map (bytes)
constexpr int oB1 = 0, oB2p = oB1 + kB1, oB2x = oB2p + kB2p;
constexpr int oL1p = oB2x + kB2x;                  // phi1 [plane][N1BUF][8] bf16
constexpr int oL1x = oL1p + 4 * N1BUF * 16;        // xi1
constexpr int oA1 = oL1x + 4 * N1BUF * 16;         // im2col [field][plane][128][8]
constexpr int oIN = oA1 + 2 * 4 * 128 * 16;        // u, v [6][IH][IW] float
constexpr int oQ = oIN + 6 * IH * IW * 4;          // q [N2][27] float
constexpr int oND = oQ + N2 * 27 * 4;              // N + D [R * WO][3] float
constexpr int oPar = oND + R * WO * 3 * 4;         // WN[96] WD[96] bL[3] outs[3] ins[6] (+pad)
constexpr int oDesc = oPar + 208 * 4;              // the tile's cloth descriptor
constexpr int oBar = oDesc + (int)sizeof(ClothDesc);   // 3 mbarriers, tensor-memory address
constexpr int kSmem = oBar + 32;
static_assert(kSmem <= 232448, "shared memory");
static_assert(oIN % 16 == 0 && oQ % 16 == 0 && oND % 16 == 0 && oPar % 16 == 0 && oDesc % 16 == 0 && oBar % 8 == 0,
              "alignment");

constexpr uint32_t kTmemCols = 256;

struct TcArgs {
    const uint4* wpack;   // packed BF16 weights (kPack bytes)
    const float* w;       // FP32 blob
    int32_t* status;
    // step mode: tiles (cloth, y0, x0, -) over the context's cloths
    const ClothDesc* desc;
    const int4* tiles;
    int n_tiles;
    const float* src;
    float* dst;
    const uint32_t* pinmask;
    // cell mode: z [N][6][H][W] -> a [N][3][H][W]
    const float* z;
    float* a;
    int N, H, W, tiles_y, tiles_x;
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&b);
}
__device__ __forceinline__ uint4 pack8(const float* v)
{
    return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}

template <bool STEP>
__global__ void __launch_bounds__(NTH, 1) net_tc_kernel(TcArgs A)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3;                 // TMEM lanes [32 quarter, +32) of this warp
    const int half = warp >> 2;                   // warps 0-3 and 4-7 split the columns
    const uint32_t sbase = tc::smem_u32(sm);
    const uint32_t bar1 = sbase + oBar, bar2[2] = {sbase + oBar + 8, sbase + oBar + 16};
    float* sIN = reinterpret_cast<float*>(sm + oIN);
    float* sQ = reinterpret_cast<float*>(sm + oQ);
    float* sND = reinterpret_cast<float*>(sm + oND);
    float* sWN = reinterpret_cast<float*>(sm + oPar);
    float* sWD = sWN + 96;
    float* sBL = sWD + 96;
    float* sOut = sBL + 3;
    float* sIns = sOut + 3;
    ClothDesc* sD = reinterpret_cast<ClothDesc*>(sm + oDesc);
    volatile uint32_t* sTmem = reinterpret_cast<uint32_t*>(sm + oBar + 24);

    // ---- one-time set-up: weights, barriers, tensor memory
    for (int e = tid; e < kPack / 16; e += NTH) reinterpret_cast<uint4*>(sm)[e] = A.wpack[e];
    for (int e = tid; e < 96; e += NTH) {
        sWN[e] = A.w[kOffWN + e];
        sWD[e] = A.w[kOffWD + e];
    }
    if (tid < 3) {
        sBL[tid] = A.w[kOffBL + tid];
        sOut[tid] = A.w[kOffOuts + tid];
    }
    if (tid < 6) sIns[tid] = A.w[kOffIns + tid];
    // rows N1 .. N1BUF of the layer-1 buffers are read only by the junk
    // positions of the last layer-2 chunk; keep them zero
    for (int e = tid; e < 2 * 4 * (N1BUF - N1); e += NTH) {
        const int buf = e / (4 * (N1BUF - N1)), rem = e % (4 * (N1BUF - N1));
        const int plane = rem / (N1BUF - N1), row = N1 + rem % (N1BUF - N1);
        reinterpret_cast<uint4*>(sm + (buf ? oL1x : oL1p))[plane * N1BUF + row] = make_uint4(0, 0, 0, 0);
    }
    if (tid == 0) {
        tc::mbar_init(bar1, 1);
        tc::mbar_init(bar2[0], 1);
        tc::mbar_init(bar2[1], 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(sbase + oBar + 24, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *sTmem;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    uint32_t ph1 = 0, ph2[2] = {0, 0};
    bool timed_out = false;
    const int n_tiles = STEP ? A.n_tiles : A.N * A.tiles_y * A.tiles_x;

    // layer-2 MMAs of chunk c into TMEM columns [128 (c & 1), +96)
    auto issue_layer2 = [&](int c2) {
        tc::fence_after();
        const uint32_t d = tmem + 128u * (uint32_t)(c2 & 1);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int row = c2 * 128 + (tap / 3) * PT + tap % 3;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool acc = tap > 0 || h > 0;
                const uint64_t ap = tc::sdesc(sbase + oL1p + (2 * h * N1BUF + row) * 16, N1BUF * 16, 128);
                const uint64_t bp = tc::sdesc(sbase + oB2p + (tap * 4 + 2 * h) * 64 * 16, 64 * 16, 128);
                tc::mma_bf16(d, ap, bp, tc::idesc_bf16(128, 64), acc);
                const uint64_t ax = tc::sdesc(sbase + oL1x + (2 * h * N1BUF + row) * 16, N1BUF * 16, 128);
                const uint64_t bx = tc::sdesc(sbase + oB2x + (tap * 4 + 2 * h) * 32 * 16, 32 * 16, 128);
                tc::mma_bf16(d + 64, ax, bx, tc::idesc_bf16(128, 32), acc);
            }
        }
        tc::mma_commit(bar2[c2 & 1]);
    };

    for (int tile = blockIdx.x; tile < n_tiles && !timed_out; tile += gridDim.x) {
        // ---- tile geometry
        int y0, x0, H, W, n = 0;
        if constexpr (STEP) {
            const int4 t = A.tiles[tile];
            if (tid == 0) *sD = A.desc[t.x];
            y0 = t.y; x0 = t.z;
            __syncthreads();
            H = sD->rows; W = sD->cols;
        } else {
            n = tile / (A.tiles_y * A.tiles_x);
            const int r = tile % (A.tiles_y * A.tiles_x);
            y0 = (r / A.tiles_x) * R; x0 = (r % A.tiles_x) * WO; H = A.H; W = A.W;
        }
        // ---- 1. input tile: u, v (raw) with a 3-node halo, zero outside the grid
        {
            int64_t cbase = 0, cstride = 0, rstride = 0;
            const float* srcp;
            if constexpr (STEP) {
                srcp = A.src + sD->plane_off; cstride = sD->plane_stride; rstride = sD->pitch;
            } else {
                srcp = A.z + (int64_t)n * 6 * H * W; cstride = (int64_t)H * W; rstride = W;
            }
            (void)cbase;
#pragma unroll 4
            for (int e = tid; e < 6 * IH * IW; e += NTH) {
                const int ch = e / (IH * IW), rem = e % (IH * IW);
                const int y = y0 - 3 + rem / IW, x = x0 - 3 + rem % IW;
                float val = 0.f;
                if (y >= 0 && y < H && x >= 0 && x < W)
                    val = __ldg(srcp + ch * cstride + (int64_t)y * rstride + (STEP ? col_pos(x) : x));
                sIN[e] = val;
            }
        }
        __syncthreads();

        // ---- 2. layer 1 (Eq. 6), chunk by chunk
        for (int c1 = 0; c1 < C1 && !timed_out; ++c1) {
            {   // im2col: thread = (field, row)
                const int row = tid & 127, f = tid >> 7;
                const int j1 = c1 * 128 + row, ry1 = j1 / PT, rx1 = j1 % PT;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int k = 8 * p + e;           // k = channel * 9 + tap
                        if (k < 27) {
                            const int ci = k / 9, tap = k % 9;
                            v[e] = sIns[3 * f + ci] *
                                   sIN[(3 * f + ci) * IH * IW + (ry1 + tap / 3) * IW + rx1 + tap % 3];
                        } else {
                            v[e] = 0.f;
                        }
                    }
                    reinterpret_cast<uint4*>(sm + oA1)[(f * 4 + p) * 128 + row] = pack8(v);
                }
            }
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after();
#pragma unroll
                for (int f = 0; f < 2; ++f)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint64_t ad = tc::sdesc(sbase + oA1 + (f * 4 + 2 * h) * 128 * 16, 128 * 16, 128);
                        const uint64_t bd = tc::sdesc(sbase + oB1 + (f * 4 + 2 * h) * 32 * 16, 32 * 16, 128);
                        tc::mma_bf16(tmem + 32 * f, ad, bd, tc::idesc_bf16(128, 32), h > 0);
                    }
                tc::mma_commit(bar1);
            }
            const bool done = tc::mbar_wait(bar1, ph1, kWaitLimit);
            ph1 ^= 1u;
            if (__syncthreads_or(!done)) { timed_out = true; break; }
            tc::fence_after();
            {   // epilogue: warp half 0 -> phi1, half 1 -> xi1; zero outside the cloth
                float r[32];
                tc::tmem_ld32(lane_base + 32 * half, r);
                tc::tmem_wait_ld();
                const int j1 = c1 * 128 + quarter * 32 + lane, ry1 = j1 / PT, rx1 = j1 % PT;
                const int y = y0 - 2 + ry1, x = x0 - 2 + rx1;
                const bool in = y >= 0 && y < H && x >= 0 && x < W;
                uint4* dstb = reinterpret_cast<uint4*>(sm + (half ? oL1x : oL1p));
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float a8[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) a8[e] = in ? r[8 * p + e] : 0.f;
                    dstb[p * N1BUF + j1] = pack8(a8);
                }
            }
            tc::fence_before();
            __syncthreads();
        }
        if (timed_out) break;
        tc::fence_async_smem();
        __syncthreads();

        // ---- 3-4. layer 2 as implicit GEMM (double-buffered in TMEM), epilogue
        if (tid == 0) issue_layer2(0);
        for (int c2 = 0; c2 < C2 && !timed_out; ++c2) {
            if (tid == 0 && c2 + 1 < C2) issue_layer2(c2 + 1);
            const int b = c2 & 1;
            const bool done = tc::mbar_wait(bar2[b], ph2[b], kWaitLimit);
            ph2[b] ^= 1u;
            if (__syncthreads_or(!done)) { timed_out = true; break; }
            tc::fence_after();
            const int j2 = c2 * 128 + quarter * 32 + lane;
            const int ry2 = j2 / PT, rx2 = j2 % PT;
            const int y = y0 - 1 + ry2, x = x0 - 1 + rx2;
            const bool valid = j2 < N2 && rx2 < WO + 2 && y >= 0 && y < H && x >= 0 && x < W;
            const uint32_t col = lane_base + 128u * (uint32_t)b;
            if (half == 1) {   // q: the WL partial sums, zero outside the cloth
                float q[32];
                tc::tmem_ld32(col + 32, q);
                tc::tmem_wait_ld();
                if (j2 < N2) {
                    float* qr = sQ + j2 * 27;
#pragma unroll
                    for (int k = 0; k < 27; ++k) qr[k] = valid ? q[k] : 0.f;
                }
            } else {           // s = tanh(t), N + D at output nodes
                float t[32], xi[32];
                tc::tmem_ld32(col + 0, t);
                tc::tmem_ld32(col + 64, xi);
                tc::tmem_wait_ld();
                const int oy = ry2 - 1, ox = rx2 - 1;
                if (valid && oy >= 0 && oy < R && ox >= 0 && ox < WO) {
                    float nd0 = 0.f, nd1 = 0.f, nd2 = 0.f;
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const float sv = tc::tanh_approx(t[c]);
                        const float xs = xi[c] * sv;
                        nd0 = fmaf(sWN[c], sv, fmaf(sWD[c], xs, nd0));
                        nd1 = fmaf(sWN[32 + c], sv, fmaf(sWD[32 + c], xs, nd1));
                        nd2 = fmaf(sWN[64 + c], sv, fmaf(sWD[64 + c], xs, nd2));
                    }
                    float* o = sND + (oy * WO + ox) * 3;
                    o[0] = nd0; o[1] = nd1; o[2] = nd2;
                }
            }
            tc::fence_before();
            __syncthreads();
        }
        if (timed_out) break;

        // ---- 5. per output node: L, a, and (step mode) the update
        for (int o = tid; o < R * WO; o += NTH) {
            const int oy = o / WO, ox = o % WO, y = y0 + oy, x = x0 + ox;
            if (y >= H || x >= W) continue;
            float acc[3];
#pragma unroll
            for (int co = 0; co < 3; ++co) {
                float L = sBL[co];
#pragma unroll
                for (int tap = 0; tap < 9; ++tap)
                    L += sQ[((oy + tap / 3) * PT + ox + tap % 3) * 27 + tap * 3 + co];
                acc[co] = sOut[co] * (L + sND[o * 3 + co]);
            }
            if constexpr (!STEP) {
#pragma unroll
                for (int co = 0; co < 3; ++co) A.a[(((int64_t)n * 3 + co) * H + y) * W + x] = acc[co];
            } else {
                const ClothDesc& D = *sD;
                const int iy = oy + 3, ix = ox + 3;
                auto U = [&](int ch, int dy, int dx) { return sIN[ch * IH * IW + (iy + dy) * IW + ix + dx]; };
                if (D.p_quarter != 0.f) {
                    const float bE = x + 1 < W ? 1.f : 0.f, bW = x > 0 ? 1.f : 0.f;
                    const float bN = y + 1 < H ? 1.f : 0.f, bS = y > 0 ? 1.f : 0.f;
                    float e[3], nn[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float ui = U(c, 0, 0);
                        e[c] = bE * (U(c, 0, 1) - ui + (c == 0 ? D.h : 0.f)) - bW * (U(c, 0, -1) - ui - (c == 0 ? D.h : 0.f));
                        nn[c] = bN * (U(c, 1, 0) - ui + (c == 1 ? D.h : 0.f)) - bS * (U(c, -1, 0) - ui - (c == 1 ? D.h : 0.f));
                    }
                    const float sc = D.p_quarter * D.inv_m;
                    acc[0] = fmaf(sc, e[1] * nn[2] - e[2] * nn[1], acc[0]);
                    acc[1] = fmaf(sc, e[2] * nn[0] - e[0] * nn[2], acc[1]);
                    acc[2] = fmaf(sc, e[0] * nn[1] - e[1] * nn[0], acc[2]);
                }
                const bool pinned = (A.pinmask[D.pin_off + (int64_t)y * D.pin_wpr + (x >> 5)] >> (x & 31)) & 1u;
                float vn[3], un[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    vn[c] = pinned ? 0.f : fmaf(D.dt, acc[c], U(3 + c, 0, 0));
                    un[c] = fmaf(D.dt, vn[c], U(c, 0, 0));
                }
                if (D.sph_on) {
                    const float rx = fmaf((float)x, D.h, -D.sph_cx) + un[0];
                    const float ry = fmaf((float)y, D.h, -D.sph_cy) + un[1];
                    const float rz = un[2] - D.sph_cz;
                    const float dd = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    if (dd < D.sph_r2 && dd > 0.f) {
                        const float sc = D.sph_r * rsqrtf(dd);
                        un[0] = fmaf(sc, rx, un[0] - rx);
                        un[1] = fmaf(sc, ry, un[1] - ry);
                        un[2] = fmaf(sc, rz, un[2] - rz);
                        vn[0] = vn[1] = vn[2] = 0.f;
                    }
                }
                if (!isfinite(un[0] + un[1] + un[2] + vn[0] + vn[1] + vn[2])) atomicOr(A.status, kStatusNonfinite);
                float* out = A.dst + D.plane_off + (int64_t)y * D.pitch + col_pos(x);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    out[c * D.plane_stride] = un[c];
                    out[(3 + c) * D.plane_stride] = vn[c];
                }
            }
        }
        __syncthreads();
    }

    // ---- tear-down: after a timeout, wait (bounded) for the MMAs in flight
    if (timed_out) {
        if (tid == 0 && A.status) atomicOr(A.status, kStatusTimeout);
        // a chunk may have been issued and not yet waited for: try both
        // phases of every barrier, each wait bounded
        for (int k = 0; k < 2; ++k) {
            tc::mbar_wait(bar1, ph1 ^ (uint32_t)k, 1u << 20);
            tc::mbar_wait(bar2[0], ph2[0] ^ (uint32_t)k, 1u << 20);
            tc::mbar_wait(bar2[1], ph2[1] ^ (uint32_t)k, 1u << 20);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// Packed BF16 B operands from the FP32 blob: one thread per row of 8 K-values.
__global__ void pack_bf16_kernel(const float* __restrict__ w, uint4* __restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int R1 = 2 * 4 * 32, R2p = 9 * 4 * 64, R2x = 9 * 4 * 32;
    if (r >= R1 + R2p + R2x) return;
    float v[8];
    if (r < R1) {   // W1 for field f: K = ci * 9 + tap over the field's 3 input channels
        const int f = r / 128, p = (r / 32) % 4, n = r % 32;
        for (int e = 0; e < 8; ++e) {
            const int k = 8 * p + e;
            v[e] = k < 27 ? w[kOffW1 + (n * 6 + 3 * f + k / 9) * 9 + k % 9] : 0.f;
        }
    } else if (r < R1 + R2p) {   // [P.W2 | WL_tap.W2] for the position field
        const int q = r - R1, tap = q / 256, p = (q / 64) % 4, n = q % 64;
        for (int e = 0; e < 8; ++e) {
            const int ci = 8 * p + e;
            float s = 0.f;
            if (n < 32) {
                for (int c = 0; c < kC; ++c) s += w[kOffP + n * kC + c] * w[kOffW2 + (c * kC + ci) * 9 + tap];
            } else if (n < 32 + 27) {
                const int m = n - 32, tl = m / 3, co = m % 3;
                for (int c = 0; c < kC; ++c) s += w[kOffWL + (co * kC + c) * 9 + tl] * w[kOffW2 + (c * kC + ci) * 9 + tap];
            }
            v[e] = s;
        }
    } else {   // W2 for the velocity field
        const int q = r - R1 - R2p, tap = q / 128, p = (q / 32) % 4, n = q % 32;
        for (int e = 0; e < 8; ++e) v[e] = w[kOffW2 + (n * kC + 8 * p + e) * 9 + tap];
    }
    out[r] = pack8(v);
}

}  // namespace

int net_tc_pack_bytes() { return kPack; }
int net_tc_tile_rows() { return R; }
int net_tc_tile_cols() { return WO; }

cudaError_t net_tc_init()
{
    cudaError_t e = cudaFuncSetAttribute(net_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(net_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    return e;
}

cudaError_t launch_pack_bf16(const float* w, void* wpack, cudaStream_t s)
{
    constexpr int rows = 2 * 4 * 32 + 9 * 4 * 64 + 9 * 4 * 32;
    pack_bf16_kernel<<<(rows + 127) / 128, 128, 0, s>>>(w, static_cast<uint4*>(wpack));
    return cudaGetLastError();
}

cudaError_t launch_net_tc_step(const void* wpack, const float* w, const ClothDesc* desc, const int4* tiles, int n_tiles,
                               const float* src, float* dst, const uint32_t* pinmask, int32_t* status, int grid,
                               cudaStream_t s)
{
    TcArgs a{};
    a.wpack = static_cast<const uint4*>(wpack);
    a.w = w;
    a.status = status;
    a.desc = desc;
    a.tiles = tiles;
    a.n_tiles = n_tiles;
    a.src = src;
    a.dst = dst;
    a.pinmask = pinmask;
    net_tc_kernel<true><<<grid, NTH, kSmem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_net_tc_forward(const void* wpack, const float* w, const float* z, float* out, int N, int H, int W,
                                  int32_t* status, int grid, cudaStream_t s)
{
    TcArgs a{};
    a.wpack = static_cast<const uint4*>(wpack);
    a.w = w;
    a.status = status;
    a.z = z;
    a.a = out;
    a.N = N; a.H = H; a.W = W;
    a.tiles_y = (H + R - 1) / R;
    a.tiles_x = (W + WO - 1) / WO;
    const int n_tiles = N * a.tiles_y * a.tiles_x;
    net_tc_kernel<false><<<grid < n_tiles ? grid : n_tiles, NTH, kSmem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace cloth
