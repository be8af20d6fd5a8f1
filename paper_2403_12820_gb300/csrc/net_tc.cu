// The CNN cell (Sec. 3.2, Eq. 6-7) and the network step (Fig. 2) fused
// into one kernel on the tcgen05 tensor cores: BF16 operands in shared
// memory, FP32 accumulators in tensor memory.
//
// One CTA (8 warps) per SM loops over tiles of R x WO output nodes.  Every
// layer region of a tile is stored at the pitch PT = WO + 6, so node
// (ry, rx) of a region has the linear index ry * PT + rx, an M = 128 MMA
// covers 128 consecutive linear indices ("a chunk"), and a 3x3 tap (ky, kx)
// is the same buffer shifted by ky * PT + kx rows — a descriptor offset,
// never a copy (implicit GEMM).  Per tile:
//   1. stage u, v of the (R+6)-row input region as BF16, 8 channels per
//      node and field (in_scale u | 0, in_scale v | 0);
//   2. layer 1 (Eq. 6): per chunk and field, 5 MMAs of K = 16, each pairing
//      two taps (the second core-matrix column of K sits LBO = the taps'
//      row distance further) against W1[:, field] -> phi1, xi1 (BF16, zero
//      outside the cloth), K-major core-matrix layout;
//   3. layer 2: per chunk and tap two MMAs of K = 16 over the shifted
//      layer-1 buffers.  The position field multiplies by
//      [P.W2 | WL_tap.W2] (N = 64): it yields t = P phi (the pre-activation
//      of s) and the 27 partial sums q_tap,co = sum_c WL[co][c][tap] phi_c
//      directly, since phi enters Eq. 7 only linearly through P and WL; the
//      velocity field multiplies by W2 (N = 32) -> xi.  Accumulators are
//      double-buffered in tensor memory so chunk c+1 runs during the
//      epilogue of chunk c;
//   4. epilogue per layer-2 node: s = tanh(t), N + D = WN s + WD (xi . s),
//      q kept in smem (zero outside the cloth: WL's zero padding);
//   5. per output node: L = bL + sum_tap q_tap at the tap's neighbour,
//      a = out_scale (L + N + D); then (step mode) v <- C(v + dt (a + f_p /
//      m)), u <- u + dt v, sphere contact, store.
// Tiles are pipelined: the input of tile t+1 is staged (into the other FP32
// tile buffer) while the layer-2 MMAs of tile t run, and the final pass of
// tile t runs while the layer-1 MMAs of tile t+1 do.
// Every wait on the tensor cores is bounded; a timeout sets a status bit
// and the kernel returns after releasing its tensor memory.
#include <cuda_bf16.h>

#include "net_internal.cuh"
#include "tc_ptx.cuh"

namespace cloth {
namespace {

constexpr int R = 12, WO = 28, PT = WO + 6;   // output rows, output columns, region pitch
constexpr int N0 = (R + 6) * PT;                // input-region nodes of a tile
constexpr int N1 = (R + 4) * PT;                // layer-1 region
constexpr int N2 = (R + 2) * PT;                // layer-2 region
constexpr int C1 = (N1 + 127) / 128;            // layer-1 chunks
constexpr int C2 = (N2 + 127) / 128;            // layer-2 chunks
constexpr int N1BUF = (C2 * 128 + 2 * PT + 2 + 15) / 16 * 16;   // layer-1 rows layer 2 reads
constexpr int N0BUF = (C1 * 128 + 2 * PT + 3 + 15) / 16 * 16;   // input rows layer 1 reads
constexpr int NWORK = 256;                       // 8 worker warps; warps w and w + 4 share TMEM lanes
constexpr int NTH = NWORK + 32;                  // + 1 warp that issues the MMAs
constexpr uint32_t kWaitLimit = 1u << 24;
static_assert(N1BUF >= N1 && N0BUF >= N0, "buffers");

// Layer-1 tap pairs: MMA p covers taps kPairA[p] and kPairB[p] (-1: none).
__host__ __device__ constexpr int pair_a(int p) { return 2 * p; }
__host__ __device__ constexpr int pair_b(int p) { return p < 4 ? 2 * p + 1 : -1; }
__host__ __device__ constexpr int tap_off(int t) { return (t / 3) * PT + t % 3; }

// packed BF16 weights: B1 [pair 5][khalf 2][64][8] (khalf = the pair's
// first / second tap; n < 32 -> phi1 from input channels 0..2 (u),
// n >= 32 -> xi1 from channels 3..5 (v)), B2p [tap][plane][64][8],
// B2x [tap][plane][32][8] (plane = 8 input channels)
constexpr int kB1 = 5 * 2 * 64 * 16, kB2p = 9 * 4 * 64 * 16, kB2x = 9 * 4 * 32 * 16;
constexpr int kPack = kB1 + kB2p + kB2x;

// FP32 u, v of the output nodes and their 1-node halo, for the update
constexpr int UH = R + 2, UW = WO + 2;
// q is kept for the valid layer-2 positions only: (R+2) x (WO+2), one plane
// per value
constexpr int NQ = (R + 2) * (WO + 2);

// shared memory map (bytes)
constexpr int oB1 = 0, oB2p = oB1 + kB1, oB2x = oB2p + kB2p;
constexpr int oIn = oB2x + kB2x;                    // input [N0BUF][8] bf16: in_scale (u, v), 0, 0
constexpr int oL1p = oIn + N0BUF * 16;              // phi1 [plane][N1BUF][8] bf16
constexpr int oL1x = oL1p + 4 * N1BUF * 16;         // xi1
constexpr int oQ = oL1x + 4 * N1BUF * 16;           // q [27][NQ] float
constexpr int kUFloats = 6 * UH * UW;
constexpr int oU = oQ + NQ * 27 * 4;                // u, v [2 tiles][6][UH][UW] float
constexpr int oND = oU + 2 * kUFloats * 4;          // N + D [R * WO][3] float (both channel halves added)
constexpr int oPar = oND + R * WO * 3 * 4;          // WND[32][8] (WN0..2 WD0..2 0 0), bL[3] outs[3] ins[6]
constexpr int oDesc = oPar + (256 + 16) * 4;        // the two tiles' cloth descriptors
constexpr int oPin = oDesc + 2 * (int)sizeof(ClothDesc);   // pinned flags of the two tiles' output nodes
constexpr int oBar = oPin + (2 * R * WO + 15) / 16 * 16;   // mbarriers: layer 1 [C1], layer 2 [2]; TMEM address
constexpr int kNumBars = C1 + 2;
constexpr int oTmemSlot = oBar + 8 * kNumBars;
constexpr int kSmem = oTmemSlot + 16;
static_assert(kSmem <= 232448, "shared memory");
static_assert(oIn % 16 == 0 && oL1p % 16 == 0 && oQ % 16 == 0 && oU % 16 == 0 && oND % 16 == 0 &&
                  oPar % 16 == 0 && oDesc % 16 == 0 && oBar % 8 == 0,
              "alignment");

// TMEM columns: layer-1 chunk c at [64 c, +64); layer-2 buffer b at
// [kL2Col + 96 b, +96)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kL2Col = 64 * C1;
static_assert(kL2Col + 2 * 96 <= kTmemCols, "tensor memory columns");

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
    const int32_t* mode;  // if set, only cloths in network mode are stepped
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool STEP>
__global__ void __launch_bounds__(NTH, 1) net_tc_kernel(TcArgs A)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = tid < NWORK, issuer = tid == NWORK;
    const int quarter = warp & 3;                 // TMEM lanes [32 quarter, +32) of this warp
    const int half = (warp >> 2) & 1;             // worker warps 0-3 and 4-7 split the columns
    const uint32_t sbase = tc::smem_u32(sm);
    float* sQ = reinterpret_cast<float*>(sm + oQ);
    float* sU = reinterpret_cast<float*>(sm + oU);
    float* sND = reinterpret_cast<float*>(sm + oND);
    const float4* sWND = reinterpret_cast<const float4*>(sm + oPar);   // [c][2]
    float* sPar = reinterpret_cast<float*>(sm + oPar);
    float* sBL = sPar + 256;
    float* sOut = sBL + 3;
    float* sIns = sOut + 3;
    ClothDesc* sD = reinterpret_cast<ClothDesc*>(sm + oDesc);
    uint8_t* sPin = sm + oPin;
    volatile uint32_t* sTmem = reinterpret_cast<uint32_t*>(sm + oTmemSlot);
    auto bar1 = [&](int c) { return sbase + oBar + 8u * (uint32_t)c; };
    auto bar2 = [&](int b) { return sbase + oBar + 8u * (uint32_t)(C1 + b); };

    // ---- one-time set-up: weights, barriers, tensor memory
    for (int e = tid; e < kPack / 16; e += NTH) reinterpret_cast<uint4*>(sm)[e] = A.wpack[e];
    for (int e = tid; e < 32 * 8; e += NTH) {
        const int c = e >> 3, j = e & 7;
        sPar[e] = j < 3 ? A.w[kOffWN + j * kC + c] : (j < 6 ? A.w[kOffWD + (j - 3) * kC + c] : 0.f);
    }
    if (tid < 3) {
        sBL[tid] = A.w[kOffBL + tid];
        sOut[tid] = A.w[kOffOuts + tid];
    }
    if (tid < 6) sIns[tid] = A.w[kOffIns + tid];
    for (int e = tid; e < R * WO * 3; e += NTH) sND[e] = 0.f;
    // input rows N0 .. N0BUF are read only by junk layer-1 positions; keep them zero
    for (int e = tid; e < N0BUF - N0; e += NTH) reinterpret_cast<uint4*>(sm + oIn)[N0 + e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int b = 0; b < kNumBars; ++b) tc::mbar_init(sbase + oBar + 8u * (uint32_t)b, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(sbase + oTmemSlot, kTmemCols);
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

    // Descriptors of the issuer: a descriptor plus (byte offset >> 4) is the
    // same matrix shifted by that offset (the start-address field is the low
    // 14 bits and every operand lies below 256 KB).
    const uint64_t dIn0 = tc::sdesc(sbase + oIn, 16, 128), dIn1 = tc::sdesc(sbase + oIn, 512, 128);
    const uint64_t dB1 = tc::sdesc(sbase + oB1, 64 * 16, 128);
    const uint64_t dL1p = tc::sdesc(sbase + oL1p, N1BUF * 16, 128), dL1x = tc::sdesc(sbase + oL1x, N1BUF * 16, 128);
    const uint64_t dB2p = tc::sdesc(sbase + oB2p, 64 * 16, 128), dB2x = tc::sdesc(sbase + oB2x, 32 * 16, 128);

    auto issue_layer1 = [&]() {   // all chunks at once, chunk c into columns [64 c, +64)
        tc::fence_after();
        for (int c1 = 0; c1 < C1; ++c1) {
#pragma unroll
            for (int p = 0; p < 5; ++p) {
                const int ta = pair_a(p), tb = pair_b(p);
                const uint64_t base = (tb >= 0 && tap_off(tb) - tap_off(ta) != 1) ? dIn1 : dIn0;
                const uint64_t ad = base + (uint64_t)(c1 * 128 + tap_off(ta));
                const uint64_t bd = dB1 + (uint64_t)(p * 2 * 64);
                tc::mma_bf16(tmem + 64u * (uint32_t)c1, ad, bd, tc::idesc_bf16(128, 64), p > 0);
            }
            tc::mma_commit(bar1(c1));
        }
    };
    auto issue_layer2 = [&](int c2) {   // chunk c2 into buffer c2 & 1
        tc::fence_after();
        const uint32_t d = tmem + kL2Col + 96u * (uint32_t)(c2 & 1);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int row = c2 * 128 + tap_off(tap);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool acc = tap > 0 || h > 0;
                const uint64_t ao = (uint64_t)(2 * h * N1BUF + row);
                tc::mma_bf16(d, dL1p + ao, dB2p + (uint64_t)((tap * 4 + 2 * h) * 64), tc::idesc_bf16(128, 64), acc);
                tc::mma_bf16(d + 64, dL1x + ao, dB2x + (uint64_t)((tap * 4 + 2 * h) * 32), tc::idesc_bf16(128, 32), acc);
            }
        }
        tc::mma_commit(bar2(c2 & 1));
    };

    // ---- per-tile pieces
    struct Geo {
        int y0, x0, H, W, n;
        const float* src;
        int64_t cs, rs;
        int cloth;
        const uint32_t* pin;   // the cloth's pin mask, pin_wpr words per row
        int pin_wpr;
    };
    auto geo = [&](int tile) {
        Geo g{};
        if constexpr (STEP) {
            const int4 t = A.tiles[tile];
            const ClothDesc& d = A.desc[t.x];
            g.cloth = t.x; g.y0 = t.y; g.x0 = t.z; g.H = d.rows; g.W = d.cols;
            g.src = A.src + d.plane_off; g.cs = d.plane_stride; g.rs = d.pitch;
            g.pin = A.pinmask + d.pin_off; g.pin_wpr = d.pin_wpr;
        } else {
            g.n = tile / (A.tiles_y * A.tiles_x);
            const int r = tile % (A.tiles_y * A.tiles_x);
            g.y0 = (r / A.tiles_x) * R; g.x0 = (r % A.tiles_x) * WO; g.H = A.H; g.W = A.W;
            g.src = A.z + (int64_t)g.n * 6 * A.H * A.W; g.cs = (int64_t)A.H * A.W; g.rs = A.W;
        }
        return g;
    };
    // this CTA's tiles: every gridDim.x-th, skipping cloths not in network mode
    auto skip = [&](int t) {
        if constexpr (STEP) {
            if (A.mode)
                while (t < n_tiles && A.mode[A.tiles[t].x] != kModeNet) t += gridDim.x;
        }
        return t;
    };

    // 1. the input region as BF16: node (iy, ix) at iy * PT + ix holds
    // (in_scale u, in_scale v, 0, 0), zero outside the grid; the raw u, v of
    // the output nodes and their halo also go to FP32 tile buffer `buf`, and
    // (step mode) the output nodes' pinned flags to sPin[buf].  Split into a
    // load of input node j0 into registers and its store to shared memory,
    // so the loads can be in flight while the thread waits for an MMA.
    struct Raw {
        float v[6];
        uint32_t pin;     // the node's pin-mask word; its bit is picked at the store
    };
    auto stage_load = [&](const Geo& g, int j0, Raw& rw) {
        const int iy = j0 / PT, ix = j0 % PT;
        const int y = g.y0 - 3 + iy, x = g.x0 - 3 + ix;
#pragma unroll
        for (int c = 0; c < 6; ++c) rw.v[c] = 0.f;
        rw.pin = 0;
        if (y >= 0 && y < g.H && x >= 0 && x < g.W) {
            const float* p0 = g.src + (int64_t)y * g.rs + (STEP ? col_pos(x) : x);
#pragma unroll
            for (int c = 0; c < 6; ++c) rw.v[c] = __ldg(p0 + c * g.cs);
            if constexpr (STEP) {
                const int oy = iy - 3, ox = ix - 3;
                if (oy >= 0 && oy < R && ox >= 0 && ox < WO) rw.pin = __ldg(g.pin + (int64_t)y * g.pin_wpr + (x >> 5));
            }
        }
    };
    auto stage_store = [&](const Geo& g, int buf, int j0, const Raw& rw) {
        const int iy = j0 / PT, ix = j0 % PT;
        float v[8];
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = sIns[c] * rw.v[c];
        v[6] = v[7] = 0.f;
        reinterpret_cast<uint4*>(sm + oIn)[j0] = pack8(v);
        const int uy = iy - 2, ux = ix - 2;
        if (uy >= 0 && uy < UH && ux >= 0 && ux < UW) {
            float* sUb = sU + buf * kUFloats;
#pragma unroll
            for (int c = 0; c < 6; ++c) sUb[(c * UH + uy) * UW + ux] = rw.v[c];
        }
        const int oy = iy - 3, ox = ix - 3;
        if (STEP && oy >= 0 && oy < R && ox >= 0 && ox < WO)
            sPin[buf * R * WO + oy * WO + ox] = (uint8_t)((rw.pin >> ((g.x0 + ox) & 31)) & 1u);
    };
    auto stage = [&](const Geo& g, int buf) {   // the whole region at once
        if (STEP && tid == 0) sD[buf] = A.desc[g.cloth];
        for (int j0 = tid; j0 < N0; j0 += NWORK) {
            Raw rw;
            stage_load(g, j0, rw);
            stage_store(g, buf, j0, rw);
        }
    };
    constexpr int kStageParts = (N0 + NWORK - 1) / NWORK;   // input nodes per worker
    static_assert(kStageParts <= C2, "one staging part per layer-2 chunk");

    // 2. layer 1 (Eq. 6) store: each chunk's phi1 / xi1 as BF16 as it
    // completes (workers; false on a timeout)
    auto repack = [&](const Geo& g) {
        auto put = [&](int c1, const float (&r)[32]) {
            const int j1 = c1 * 128 + quarter * 32 + lane, ry1 = j1 / PT, rx1 = j1 % PT;
            const int y = g.y0 - 2 + ry1, x = g.x0 - 2 + rx1;
            const bool in = j1 < N1 && rx1 < WO + 4 && y >= 0 && y < g.H && x >= 0 && x < g.W;
            if (j1 < N1BUF) {
                uint4* dstb = reinterpret_cast<uint4*>(sm + (half ? oL1x : oL1p));
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float a8[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) a8[e] = in ? r[8 * p + e] : 0.f;
                    dstb[p * N1BUF + j1] = pack8(a8);
                }
            }
        };
        // two chunks' tensor-memory loads in flight at a time
        for (int c1 = 0; c1 < C1; c1 += 2) {
            const bool two = c1 + 1 < C1;
            if (!tc::mbar_wait(bar1(c1), ph1, kWaitLimit)) return false;
            if (two && !tc::mbar_wait(bar1(c1 + 1), ph1, kWaitLimit)) return false;
            tc::fence_after();
            float r0[32], r1[32];
            tc::tmem_ld32(lane_base + 64u * (uint32_t)c1 + 32u * (uint32_t)half, r0);
            if (two) tc::tmem_ld32(lane_base + 64u * (uint32_t)(c1 + 1) + 32u * (uint32_t)half, r1);
            tc::tmem_wait_ld();
            put(c1, r0);
            if (two) put(c1 + 1, r1);
        }
        tc::fence_async_smem();
        tc::fence_before();
        return true;
    };

    // 4. epilogue of layer-2 chunk c2 (TMEM buffer b): s = tanh(t), N + D
    // over the channel half [16 half, +16) added into sND; q, the WL
    // partial sums, into sQ (zero outside the cloth: WL's zero padding)
    auto epilogue = [&](const Geo& g, int c2, int b) {
        tc::fence_after();
        const int j2 = c2 * 128 + quarter * 32 + lane;
        const int ry2 = j2 / PT, rx2 = j2 % PT;
        const int y = g.y0 - 1 + ry2, x = g.x0 - 1 + rx2;
        const bool valid = j2 < N2 && rx2 < WO + 2 && y >= 0 && y < g.H && x >= 0 && x < g.W;
        const int oy = ry2 - 1, ox = rx2 - 1;
        const bool out_node = valid && oy >= 0 && oy < R && ox >= 0 && ox < WO;
        const uint32_t col = lane_base + kL2Col + 96u * (uint32_t)b;
        float t[16], xi[16], q[16];
        tmem_ld16(col + 16 * half, t);
        tmem_ld16(col + 64 + 16 * half, xi);
        tmem_ld16(col + 32 + 16 * half, q);   // q_0..15 (half 0) or q_16..26 and padding (half 1)
        tc::tmem_wait_ld();
        if (j2 < N2 && rx2 < WO + 2) {
            float* qr = sQ + 16 * half * NQ + ry2 * (WO + 2) + rx2;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < 11 || half == 0) qr[k * NQ] = valid ? q[k] : 0.f;
        }
        if (out_node) {
            float nd0 = 0.f, nd1 = 0.f, nd2 = 0.f;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const float sv = tc::tanh_approx(t[c]);
                const float xs = xi[c] * sv;
                const float4 w0 = sWND[2 * (16 * half + c)], w1 = sWND[2 * (16 * half + c) + 1];
                nd0 = fmaf(w0.x, sv, fmaf(w0.w, xs, nd0));
                nd1 = fmaf(w0.y, sv, fmaf(w1.x, xs, nd1));
                nd2 = fmaf(w0.z, sv, fmaf(w1.y, xs, nd2));
            }
            // the two halves' sums land on zero: x + y == y + x, so the
            // result does not depend on their order
            float* o = sND + (oy * WO + ox) * 3;
            atomicAdd(o + 0, nd0);
            atomicAdd(o + 1, nd1);
            atomicAdd(o + 2, nd2);
        }
        tc::fence_before();
    };

    // 5. per output node: L, a, and (step mode) the update; sND is zeroed
    // for the next tile (workers)
    auto final_pass = [&](const Geo& g, int buf) {
        const float* sUb = sU + buf * kUFloats;
        for (int o = tid; o < R * WO; o += NWORK) {
            const int oy = o / WO, ox = o % WO, y = g.y0 + oy, x = g.x0 + ox;
            float acc[3];
#pragma unroll
            for (int co = 0; co < 3; ++co) {
                float L = sBL[co];
#pragma unroll
                for (int tap = 0; tap < 9; ++tap)
                    L += sQ[(tap * 3 + co) * NQ + (oy + tap / 3) * (WO + 2) + ox + tap % 3];
                acc[co] = sOut[co] * (L + sND[o * 3 + co]);
                sND[o * 3 + co] = 0.f;
            }
            if (y >= g.H || x >= g.W) continue;
            if constexpr (!STEP) {
#pragma unroll
                for (int co = 0; co < 3; ++co) A.a[(((int64_t)g.n * 3 + co) * g.H + y) * g.W + x] = acc[co];
            } else {
                const ClothDesc& D = sD[buf];
                auto U = [&](int ch, int yy, int xx) {   // from the FP32 tile
                    return sUb[(ch * UH + yy - g.y0 + 1) * UW + xx - g.x0 + 1];
                };
                float u[3], v[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    u[c] = U(c, y, x);
                    v[c] = U(3 + c, y, x);
                }
                if (D.p_quarter != 0.f) {
                    const bool bE = x + 1 < g.W, bW = x > 0, bN = y + 1 < g.H, bS = y > 0;
                    float e[3], nn[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        e[c] = (bE ? U(c, y, x + 1) - u[c] + (c == 0 ? D.h : 0.f) : 0.f) -
                               (bW ? U(c, y, x - 1) - u[c] - (c == 0 ? D.h : 0.f) : 0.f);
                        nn[c] = (bN ? U(c, y + 1, x) - u[c] + (c == 1 ? D.h : 0.f) : 0.f) -
                                (bS ? U(c, y - 1, x) - u[c] - (c == 1 ? D.h : 0.f) : 0.f);
                    }
                    const float sc = D.p_quarter * D.inv_m;
                    acc[0] = fmaf(sc, e[1] * nn[2] - e[2] * nn[1], acc[0]);
                    acc[1] = fmaf(sc, e[2] * nn[0] - e[0] * nn[2], acc[1]);
                    acc[2] = fmaf(sc, e[0] * nn[1] - e[1] * nn[0], acc[2]);
                }
                const bool pinned = sPin[buf * R * WO + o] != 0;
                float vn[3], un[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    vn[c] = pinned ? pin_v(D, c) : fmaf(D.dt_net, acc[c], v[c]);
                    un[c] = fmaf(D.dt_net, vn[c], u[c]);
                }
                if (D.sph_on) sphere_contact(D, x, y, D.h, un[0], un[1], un[2], vn[0], vn[1], vn[2]);
                if (!isfinite(un[0] + un[1] + un[2] + vn[0] + vn[1] + vn[2])) atomicOr(A.status, kStatusNonfinite);
                float* out = A.dst + D.plane_off + (int64_t)y * D.pitch + col_pos(x);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    out[c * D.plane_stride] = un[c];
                    out[(3 + c) * D.plane_stride] = vn[c];
                }
            }
        }
    };

    // ---- the pipeline.  Prologue: stage and run layer 1 of the first tile.
    // The geometry of the tile after the current one is known one iteration
    // ahead, so its loads have landed when its input is fetched.
    int tile = skip((int)blockIdx.x);
    int buf = 0;
    Geo g{}, gn{};
    int tn = n_tiles;
    if (tile < n_tiles) {
        g = geo(tile);
        tn = skip(tile + (int)gridDim.x);
        if (tn < n_tiles) gn = geo(tn);
        if (worker) {
            stage(g, 0);
            tc::fence_async_smem();
        }
        __syncthreads();
        if (issuer) issue_layer1();
        bool ok = true;
        if (worker) ok = repack(g);
        ph1 ^= 1u;
        if (__syncthreads_or(!ok)) timed_out = true;
    }
    while (tile < n_tiles && !timed_out) {
        const bool has_next = tn < n_tiles;

        // 3-4. layer 2 of this tile as implicit GEMM, double-buffered in TMEM
        // (chunk c+1 runs while the workers read chunk c).  Each worker loads
        // its input nodes of the next tile up front and stores one after each
        // of the first chunks' epilogues, so the loads have the MMAs' time to
        // land.
        if (issuer) {
            issue_layer2(0);
            if (C2 > 1) issue_layer2(1);
        }
        Raw rw[kStageParts];
        if (worker && has_next) {
#pragma unroll
            for (int k = 0; k < kStageParts; ++k)
                if (tid + k * NWORK < N0) stage_load(gn, tid + k * NWORK, rw[k]);
        }
        // the next tile's descriptor (8 x 16 bytes), stored after chunk 0
        constexpr int kDescV = (int)(sizeof(ClothDesc) / sizeof(uint4));
        static_assert(sizeof(ClothDesc) % sizeof(uint4) == 0 && kDescV <= NWORK, "descriptor copy");
        uint4 dv = make_uint4(0, 0, 0, 0);
        if (STEP && has_next && tid < kDescV) dv = reinterpret_cast<const uint4*>(A.desc + gn.cloth)[tid];
        // the tile after next: its geometry loads land during the chunks
        const int tnn = has_next ? skip(tn + (int)gridDim.x) : n_tiles;
        Geo gnn{};
        if (tnn < n_tiles) gnn = geo(tnn);
        for (int c2 = 0; c2 < C2; ++c2) {
            const int b = c2 & 1;
            bool ok = true;
            if (worker) {
                ok = tc::mbar_wait(bar2(b), ph2[b], kWaitLimit);
                if (ok) epilogue(g, c2, b);
#pragma unroll
                for (int k = 0; k < kStageParts; ++k)   // register-indexed: k is a constant here
                    if (k == c2 && has_next && tid + k * NWORK < N0) stage_store(gn, buf ^ 1, tid + k * NWORK, rw[k]);
                if (STEP && c2 == 0 && has_next && tid < kDescV) reinterpret_cast<uint4*>(sD + (buf ^ 1))[tid] = dv;
            }
            ph2[b] ^= 1u;
            if (__syncthreads_or(!ok)) { timed_out = true; break; }
            if (issuer && c2 + 2 < C2) issue_layer2(c2 + 2);   // buffer b is free again
        }
        if (timed_out) break;

        // layer 1 of the next tile runs during this tile's final pass
        if (worker) tc::fence_async_smem();   // the staged input, for the tensor cores
        __syncthreads();
        if (issuer && has_next) issue_layer1();
        bool ok = true;
        if (worker) {
            final_pass(g, buf);
            if (has_next) ok = repack(gn);
        }
        if (has_next) ph1 ^= 1u;
        if (__syncthreads_or(!ok)) { timed_out = true; break; }
        tile = tn;
        tn = tnn;
        g = gn;
        gn = gnn;
        buf ^= 1;
    }

    // ---- tear-down: after a timeout, wait (bounded) for the MMAs in flight
    // (a chunk may have been issued and not yet waited for: try both phases)
    if (timed_out) {
        if (tid == 0 && A.status) atomicOr(A.status, kStatusTimeout);
        for (int k = 0; k < 2; ++k)
            for (int b = 0; b < kNumBars; ++b)
                tc::mbar_wait(sbase + oBar + 8u * (uint32_t)b, (uint32_t)k, 1u << 18);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// Packed BF16 B operands from the FP32 blob: one thread per row of 8 K-values.
__global__ void pack_bf16_kernel(const float* __restrict__ w, uint4* __restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int R1 = 5 * 2 * 64, R2p = 9 * 4 * 64, R2x = 9 * 4 * 32;
    if (r >= R1 + R2p + R2x) return;
    float v[8];
    if (r < R1) {   // W1: tap pair p, the pair's first (kh 0) or second tap; n < 32 phi1 from
                    // u (channels 0..2 of a node), n >= 32 xi1 from v (channels 3..5)
        const int p = r / 128, kh = (r / 64) % 2, n = r % 64;
        const int tap = kh == 0 ? pair_a(p) : pair_b(p);
        const int f = n / 32, co = n % 32;
        for (int e = 0; e < 8; ++e)
            v[e] = (tap >= 0 && e / 3 == f && e < 6) ? w[kOffW1 + (co * 6 + e) * 9 + tap] : 0.f;
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
    constexpr int rows = 5 * 2 * 64 + 9 * 4 * 64 + 9 * 4 * 32;
    pack_bf16_kernel<<<(rows + 127) / 128, 128, 0, s>>>(w, static_cast<uint4*>(wpack));
    return cudaGetLastError();
}

cudaError_t launch_net_tc_step(const void* wpack, const float* w, const ClothDesc* desc, const int4* tiles, int n_tiles,
                               const float* src, float* dst, const uint32_t* pinmask, int32_t* status, int grid,
                               cudaStream_t s, const int32_t* mode)
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
    a.mode = mode;
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
