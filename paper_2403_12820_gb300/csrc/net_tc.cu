// The CNN cell (Sec. 3.2, Eq. 6-7) and the network step (Fig. 2) fused
// into one kernel on the tcgen05 tensor cores: BF16 operands in shared
// memory, FP32 accumulators in tensor memory.
//
// The trunk W2 (*) (W1 (*) z) is linear and bias-free, and its output phi
// enters Eq. 7 only through P (the nonlinear branches) and WL (the linear
// branch).  Away from the cloth's edge the two 3x3 convolutions are one
// 5x5 convolution with the composite kernel C_c = sum_{a+b=c} W2_a W1_b,
// so the kernel evaluates per node, in one implicit GEMM,
//   t = P C (*) u   (the pre-activation of s),
//   q_tap = WL_tap C (*) u   (27 partial sums of the linear branch),
//   xi = C (*) v   (the velocity features),
// an MMA of N = 96 output columns per 128 nodes.  The layers' zero padding
// makes the composite differ from the layered trunk only on the cloth's
// outermost ring of nodes: there the terms through the layer-1 positions
// outside the cloth are removed again (a 5-tap correction per edge the node
// lies on, with a single-tap add-back where two edges meet), in FP32 from
// the same BF16 inputs, so every node gets the layered result.
//
// One CTA (16 worker warps, 1 warp that issues the MMAs and 3 helper warps)
// per SM loops over tiles of R x WO output nodes.  Every region of a tile is stored at the
// pitch PT = WO + 6, so node (ry, rx) of a region has the linear index
// ry * PT + rx, an M = 128 MMA covers 128 consecutive linear indices ("a
// chunk"), and a 5x5 tap (cy, cx) is the same buffer shifted by
// cy * PT + cx rows — a descriptor offset, never a copy.  Per tile:
//   1. stage u, v of the (R+6)-row input region as BF16 (in_scale u,
//      in_scale v, 0, 0 per node; zero outside the cloth) into one of two
//      input buffers, and the raw FP32 u, v of the output nodes and their
//      1-node halo into one of two FP32 tile buffers;
//   2. per chunk of the (R+2)-row cell region (R = 14, 10 or 6 with
//      WO = 26: exactly four, three or two chunks), 13 MMAs of K = 16, each
//      pairing two of the 25 taps (the second core-matrix column of K sits
//      LBO = the taps' row distance further), into one of two tensor-memory accumulators (chunk c+1 runs
//      during the epilogue of chunk c);
//   3. epilogue per cell-region node: the edge corrections (computed per
//      tile from the staged input, before its first epilogue), s = tanh(t)
//      and xi . s as the BF16 A operand of a second MMA, N + D = [s, xi . s]
//      [WN | WD]^T (M = 128, N = 16, K = 64) into a third tensor-memory
//      region; q kept in shared memory (zero outside the cloth: WL's zero
//      padding);
//   4. per cell-region node that is an output node (one thread each: the
//      16 worker warps are the region's 16 rows): L = bL + sum_tap q_tap at
//      the tap's neighbour, N + D from tensor memory, a = out_scale (L + N +
//      D); then (step mode) v <- C(v + dt (a + f_p / m)), u <- u + dt v,
//      sphere contact, store.
// Tiles are pipelined: the helper warps stage the input of tile t+1 (step
// 1, with its tile entry and cloth descriptor, from which the workers take
// its geometry without a global load) while the chunks of tile t run, and
// the first two chunks of tile t+1 run during the final pass of tile t.
// Between the chunks there is no CTA barrier: each worker warp arrives on
// an accumulator's "free" mbarrier once it has read it, and the issuing
// thread waits there before it reuses the accumulator; a tile has two CTA
// barriers (before and after its final pass).  Every wait on the tensor
// cores is bounded; a timeout sets a status bit and the kernel returns after
// releasing its tensor memory.
#include <cuda_bf16.h>

#include "net_internal.cuh"
#include "tc_ptx.cuh"

namespace cloth {
namespace {

constexpr int WO = 26, PT = WO + 6;              // output columns, region pitch
constexpr int NWORK = 512;                       // 16 worker warps; warps w, w + 4, w + 8, w + 12 share TMEM lanes
constexpr int NHELP = 96;                        // 3 helper warps: stage the next tile's input
constexpr int NTH = NWORK + 32 + NHELP;          // + 1 warp that issues the MMAs + the helpers
constexpr int kNC = 96;                          // MMA N: t [0, 32), q [32, 59), 0 [59, 64), xi [64, 96)
constexpr int kPairs = 13;                       // 25 taps in K = 16 pairs (the last pair's second tap is 0)
constexpr uint32_t kWaitLimit = 1u << 24;

// composite tap c = 5 cy + cx reads the input-region row j2 + cy * PT + cx
// of cell-region node j2
__host__ __device__ constexpr int ctap_off(int c) { return (c / 5) * PT + c % 5; }

// Packed operands (bytes): BF16 B [pair 13][khalf 2][96][8] (khalf = the
// pair's first / second tap, 8 = the input slots u0 u1 u2 v0 v1 v2 0 0);
// FP32 edge corrections KE [edge 4: x = 0, x = W-1, y = 0, y = H-1][tap 5]
// [channel 3][96] and corner add-backs KC [corner 4][channel 3][96], where
// output columns below 64 take u's channels and the others v's.
constexpr int kBc = kPairs * 2 * kNC * 16;
constexpr int kKE = 4 * 5 * 3 * kNC, kKC = 4 * 3 * kNC;   // floats
// FP32 rounding defects KD [direction 2: taps (s, 2) of the x edges, taps
// (2, s) of the y edges][tap s 5][channel 3][96]: the composite tap's FP32
// value less its BF16 value in B.  An edge node keeps only part of the
// composite taps on its edge column or row, so their BF16 rounding error
// would be large against what remains (up to 9x on a 1 x 1 cloth); the edge
// terms add the defect back once per tap, which makes those taps FP32.
constexpr int kKD = 2 * 5 * 3 * kNC;
// BF16 B operand of the N + D MMA: [k / 8][n 16][k % 8], k < 32 the s
// channels (WN), k >= 32 the xi . s channels (WD); columns n >= 3 are zero.
constexpr int kNDN = 16, kNDK = 64;
constexpr int kOffBnd = kBc + (kKE + kKC + kKD) * 4;
constexpr int kBnd = kNDK * kNDN * 2;
// The three-term split of the FP32 step: B = Bhi + Blo with Bhi the BF16 B
// above and Blo = BF16(B - Bhi) in the same layout, and the defects KD2 =
// B - (Bhi + Blo) in KD's layout.
constexpr int kOffBlo = kOffBnd + kBnd;
constexpr int kOffKD2 = kOffBlo + kBc;
constexpr int kPack = kOffKD2 + kKD * 4;
static_assert(kPack % 16 == 0 && kOffBlo % 16 == 0, "pack");

constexpr int UW = WO + 2;
// an edge node's slot of the edge table: its 96 columns, padded so that the
// slots of a warp's 32 edge nodes (a y-edge row) fall on different banks
constexpr int kCorrW = kNC + 4;
constexpr int kAnd = (kNDK / 8) * 128 * 16;      // bytes of one N + D operand [8][128][8] bf16
// mbarriers: accumulator b full (MMAs done) at b, free (16 warps read it and
// wrote their part of the N + D operand) at 2 + b, the tile's N + D done at
// 4, the tear-down drain at 5; in the FP32 form, accumulator b read (16 warps
// loaded it into registers) at 6 + b
constexpr int kNumBars = 8;
// TMEM columns: accumulator b at [96 b, +96), N + D of chunk c at
// [192 + 16 c, +16)
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kTmemND = 2 * kNC;

// A tile shape: C2 chunks of 128 cell-region nodes = C2 * 4 rows of PT, so
// R = 4 C2 - 2 output rows of WO columns.  SPLIT: the FP32 step, each BF16
// operand as a high and a low part (three MMAs per product: hi hi, hi lo,
// lo hi), N + D and tanh in FP32 on the CUDA cores.
template <int C2V, bool SPLITV>
struct TcShape {
    static constexpr int C2 = C2V;
    static constexpr bool SPLIT = SPLITV;
    static constexpr int R = 4 * C2 - 2;                  // output rows
    static constexpr int N0 = (R + 6) * PT;               // input-region nodes of a tile (origin y0 - 3, x0 - 3)
    static constexpr int N2 = (R + 2) * PT;               // cell region (origin y0 - 1, x0 - 1)
    static constexpr int N0BUF = (C2 * 128 + 4 * PT + 4 + 1 + 15) / 16 * 16;   // input rows the MMAs read
    static constexpr int kParts = SPLIT ? 2 : 1;          // BF16 parts of each operand
    // FP32 u, v of the output nodes and their 1-node halo, for the update
    static constexpr int UH = R + 2;
    // q is kept for the valid cell-region positions only: (R+2) x (WO+2),
    // one plane per value
    static constexpr int NQ = (R + 2) * (WO + 2);
    static constexpr int kSlots = 2 * (R + 2) + 2 * (WO + 2);   // edge nodes: x = 0, x = W-1, y = 0, y = H-1
    static constexpr int kCorr = kSlots * kCorrW;         // floats of one tile's edge table
    static constexpr int kUFloats = 6 * UH * UW;
    // shared memory map (bytes)
    static constexpr int oBc = 0;                         // B [part][pair][khalf][96][8] bf16
    static constexpr int oIn = oBc + kParts * kBc;        // input [2 tiles][part][N0BUF][8] bf16
    static constexpr int oBnd = oIn + 2 * kParts * N0BUF * 16;   // B of the N + D MMA (BF16 only)
    static constexpr int oAnd = oBnd + (SPLIT ? 0 : kBnd);       // A of the N + D MMA [2 accumulators] (BF16 only)
    static constexpr int oCorr = oAnd + (SPLIT ? 0 : 2 * kAnd);  // the edge nodes' corrections [kSlots][kCorrW] float
    static constexpr int oQ = oCorr + kCorr * 4;          // q [27][NQ] float
    // SPLIT: the N + D partial sums of the 4 channel groups [4][3][C2 * 128] float
    static constexpr int oND = oQ + NQ * 27 * 4;
    static constexpr int kNDp = SPLIT ? 4 * 3 * C2 * 128 : 0;
    static constexpr int oU = oND + kNDp * 4;             // u, v [2 tiles][6][UH][UW] float
    static constexpr int oPar = oU + 2 * kUFloats * 4;    // bL[3] outs[3] ins[6] (SPLIT: + WN[3][32], WD[3][32])
    static constexpr int kParFloats = SPLIT ? 16 + 6 * 32 : 16;
    static constexpr int oDesc = oPar + kParFloats * 4;   // the two tiles' cloth descriptors
    static constexpr int oTile = oDesc + 2 * (int)sizeof(ClothDesc);  // the two tiles' entries (cloth, y0, x0, -)
    static constexpr int oPin = oTile + 2 * 16;           // pinned flags of the two tiles' output nodes
    static constexpr int oBar = oPin + (2 * R * WO + 15) / 16 * 16;  // mbarriers; TMEM address
    static constexpr int oTmemSlot = oBar + 8 * kNumBars;
    static constexpr int kSmem = oTmemSlot + 16;
    static_assert(C2 >= 2 && C2 <= 4, "two chunks in flight; the final pass gives each worker warp one region row");
    static_assert(N0BUF >= N0 && N0BUF >= C2 * 128 + 4 * PT + 4 + 1, "input buffer");
    static_assert(kSmem <= 232448, "shared memory");
    static_assert(oIn % 16 == 0 && oBnd % 16 == 0 && oAnd % 16 == 0 && oCorr % 16 == 0 && oQ % 16 == 0 &&
                      oND % 16 == 0 && oU % 16 == 0 && oPar % 16 == 0 && oDesc % 16 == 0 && oBar % 8 == 0,
                  "alignment");
    static_assert(kTmemND + C2 * kNDN <= kTmemCols, "tensor memory columns");
};

struct TcArgs {
    const uint4* wpack;   // packed operands (kPack bytes)
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
__device__ __forceinline__ float bf_lo(uint32_t x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf_hi(uint32_t x) { return __uint_as_float(x & 0xffff0000u); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool STEP, int C2V, bool SPLIT>
__global__ void __launch_bounds__(NTH, 1) net_tc_kernel(TcArgs A)
{
    using S = TcShape<C2V, SPLIT>;
    constexpr int C2 = S::C2, R = S::R, N0 = S::N0, N2 = S::N2, N0BUF = S::N0BUF, kParts = S::kParts;
    constexpr int UH = S::UH, NQ = S::NQ, kUFloats = S::kUFloats;
    constexpr int oBc = S::oBc, oIn = S::oIn, oBnd = S::oBnd, oAnd = S::oAnd, oCorr = S::oCorr, oQ = S::oQ;
    constexpr int oND = S::oND, oU = S::oU, oPar = S::oPar, oDesc = S::oDesc, oTile = S::oTile, oPin = S::oPin;
    constexpr int oBar = S::oBar;
    constexpr int oTmemSlot = S::oTmemSlot;
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = tid < NWORK, issuer = tid == NWORK, helper = tid >= NWORK + 32;
    const int htid = tid - (NWORK + 32);          // helper thread index
    const int quarter = warp & 3;                 // TMEM lanes [32 quarter, +32) of this warp
    const int cg = (warp >> 2) & 3;               // channel group: columns [8 cg, +8) of t, q and xi
    const uint32_t sbase = tc::smem_u32(sm);
    // the FP32 edge and corner terms stay in global memory (read once per
    // edge tile, through the L1 cache)
    const float* gKE = reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(A.wpack) + kBc);
    const float* gKC = gKE + kKE;
    auto sCorr = [&](int) { return reinterpret_cast<float*>(sm + oCorr); };   // one edge table for both tile buffers
    float* sQ = reinterpret_cast<float*>(sm + oQ);
    float* sU = reinterpret_cast<float*>(sm + oU);
    float* sPar = reinterpret_cast<float*>(sm + oPar);
    float* sBL = sPar;
    float* sOut = sBL + 3;
    float* sIns = sOut + 3;
    float* sNDW = sPar + 16;   // SPLIT: WN [3][32], then WD [3][32]
    float* sND = reinterpret_cast<float*>(sm + oND);   // SPLIT: N + D partial sums [channel group 4][3][C2 * 128]
    ClothDesc* sD = reinterpret_cast<ClothDesc*>(sm + oDesc);
    int4* sTile = reinterpret_cast<int4*>(sm + oTile);
    uint8_t* sPin = sm + oPin;
    volatile uint32_t* sTmem = reinterpret_cast<uint32_t*>(sm + oTmemSlot);
    auto bar = [&](int b) { return sbase + oBar + 8u * (uint32_t)b; };
    auto bar_free = [&](int b) { return sbase + oBar + 8u * (uint32_t)(2 + b); };
    const uint32_t bar_nd = sbase + oBar + 8u * 4u, bar_drain = sbase + oBar + 8u * 5u;
    auto bar_read = [&](int b) { return sbase + oBar + 8u * (uint32_t)(6 + b); };
    // input buffer of tile buffer `buf` (SPLIT: its high part; the low part follows at + N0BUF)
    auto sIn = [&](int buf, int part = 0) { return reinterpret_cast<uint4*>(sm + oIn) + (buf * kParts + part) * N0BUF; };

    // ---- one-time set-up: operands, barriers, tensor memory
    for (int e = tid; e < kBc / 16; e += NTH) reinterpret_cast<uint4*>(sm + oBc)[e] = A.wpack[e];
    if constexpr (SPLIT) {
        for (int e = tid; e < kBc / 16; e += NTH) reinterpret_cast<uint4*>(sm + oBc + kBc)[e] = A.wpack[kOffBlo / 16 + e];
        for (int e = tid; e < 6 * kC; e += NTH) sNDW[e] = A.w[(e < 3 * kC ? kOffWN : kOffWD) + e % (3 * kC)];
    } else {
        for (int e = tid; e < kBnd / 16; e += NTH) reinterpret_cast<uint4*>(sm + oBnd)[e] = A.wpack[kOffBnd / 16 + e];
    }
    if (tid < 3) {
        sBL[tid] = A.w[kOffBL + tid];
        sOut[tid] = A.w[kOffOuts + tid];
    }
    if (tid < 6) sIns[tid] = A.w[kOffIns + tid];
    // input rows N0 .. N0BUF are read only by junk cell-region positions; keep them zero
    for (int e = tid; e < 2 * kParts * (N0BUF - N0); e += NTH) {
        const int bp = e / (N0BUF - N0);
        sIn(bp / kParts, bp % kParts)[N0 + e % (N0BUF - N0)] = make_uint4(0, 0, 0, 0);
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(bar(b), 1);
            tc::mbar_init(bar_free(b), NWORK / 32);
        }
        tc::mbar_init(bar_nd, 1);
        tc::mbar_init(bar_drain, 1);
        for (int b = 0; b < 2; ++b) tc::mbar_init(bar_read(b), NWORK / 32);
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
    uint32_t ph = 0;      // bit b: the workers' phase of accumulator b's barrier
    uint32_t ph_nd = 0;   // the workers' phase of bar_nd (one completion per tile)
    bool timed_out = false;
    const int n_tiles = STEP ? A.n_tiles : A.N * A.tiles_y * A.tiles_x;

    // Descriptors of the issuer: a descriptor plus (byte offset >> 4) is the
    // same matrix shifted by that offset (the start-address field is the low
    // 14 bits and every operand lies below 256 KB).  Taps in one row pair at
    // LBO = 16 bytes, a row's last tap with the next row's first at LBO =
    // (PT - 4) rows.
    const uint64_t dBc = tc::sdesc(sbase + oBc, kNC * 16, 128);
    // N + D operands: A [k / 8][row 128][8] (LBO 128 rows, SBO 8 rows), B
    // [k / 8][n 16][8] (LBO 16 rows, SBO 8 rows); one MMA per 16 of K
    const uint64_t dBnd = tc::sdesc(sbase + oBnd, kNDN * 16, 128);
    // the issuer's view of the accumulators: it waits on an accumulator's
    // "free" barrier (the 16 worker warps read it and wrote their part of the
    // N + D operand) before it issues that chunk's N + D MMA and reuses the
    // accumulator
    uint32_t pfree = 0;   // bit b: the issuer's phase of accumulator b's free barrier
    auto wait_free = [&](int b) {
        if (!tc::mbar_wait(bar_free(b), (pfree >> b) & 1u, kWaitLimit)) return false;
        pfree ^= 1u << b;
        tc::fence_after();
        return true;
    };
    uint32_t pread = 0;   // bit b: the issuer's phase of accumulator b's read barrier (FP32 form)
    auto wait_read = [&](int b) {
        if (!tc::mbar_wait(bar_read(b), (pread >> b) & 1u, kWaitLimit)) return false;
        pread ^= 1u << b;
        tc::fence_after();
        return true;
    };
    auto issue_nd = [&](int c2) {   // N + D of chunk c2 from A operand c2 & 1
        const uint32_t d = tmem + kTmemND + (uint32_t)(kNDN * c2);
        const uint64_t dA = tc::sdesc(sbase + oAnd + (uint32_t)((c2 & 1) * kAnd), 128 * 16, 128);
#pragma unroll
        for (int k = 0; k < kNDK / 16; ++k)
            tc::mma_bf16(d, dA + (uint64_t)(k * 2 * 128), dBnd + (uint64_t)(k * 2 * kNDN), tc::idesc_bf16(128, kNDN), k > 0);
    };
    auto issue_chunk = [&](int c2, int ib) {   // chunk c2 of input buffer ib into accumulator c2 & 1
        const uint32_t d = tmem + (uint32_t)kNC * (uint32_t)(c2 & 1);
        const uint32_t in = sbase + oIn + (uint32_t)(ib * kParts * N0BUF * 16);
        const uint64_t dA = tc::sdesc(in, 16, 128), dAw = tc::sdesc(in, (PT - 4) * 16, 128);
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
            const int ta = 2 * p;
            const bool wrap = p < kPairs - 1 && ta % 5 == 4;
            const uint64_t ad = (wrap ? dAw : dA) + (uint64_t)(c2 * 128 + ctap_off(ta));
            tc::mma_bf16(d, ad, dBc + (uint64_t)(p * 2 * kNC), tc::idesc_bf16(128, kNC), p > 0);
            if constexpr (SPLIT) {   // + A_hi B_lo + A_lo B_hi (the low parts sit kBc and N0BUF rows further)
                tc::mma_bf16(d, ad, dBc + (uint64_t)(kBc >> 4) + (uint64_t)(p * 2 * kNC), tc::idesc_bf16(128, kNC), true);
                tc::mma_bf16(d, ad + (uint64_t)N0BUF, dBc + (uint64_t)(p * 2 * kNC), tc::idesc_bf16(128, kNC), true);
            }
        }
        tc::mma_commit(bar(c2 & 1));
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
    // the same from the copies in shared memory of tile buffer b (step mode:
    // the tile's entry and its cloth's descriptor, staged with its input),
    // so the workers start a tile without a dependent global load
    auto geo_s = [&](int tile, int b) {
        if constexpr (STEP) {
            const int4 t = sTile[b];
            const ClothDesc& d = sD[b];
            Geo g{};
            g.cloth = t.x; g.y0 = t.y; g.x0 = t.z; g.H = d.rows; g.W = d.cols;
            g.src = A.src + d.plane_off; g.cs = d.plane_stride; g.rs = d.pitch;
            g.pin = A.pinmask + d.pin_off; g.pin_wpr = d.pin_wpr;
            return g;
        } else {
            return geo(tile);
        }
    };
    // this CTA's tiles: every gridDim.x-th, skipping cloths not in network mode
    auto skip = [&](int t) {
        if constexpr (STEP) {
            if (A.mode)
                while (t < n_tiles && A.mode[A.tiles[t].x] != kModeNet) t += gridDim.x;
        }
        return t;
    };

    // 1. the input region as BF16: node (iy, ix) at iy * PT + ix of input
    // buffer `buf` holds (in_scale u, in_scale v, 0, 0), zero outside the
    // grid; the raw u, v of the output nodes and their halo also go to FP32
    // tile buffer `buf`, and (step mode) the output nodes' pinned flags to
    // sPin[buf].  Split into a load of input node j0 into registers and its
    // store to shared memory, so that a helper has all its nodes' loads in
    // flight at once.
    struct Raw {
        float v[6];
        uint32_t pin;     // the node's pin-mask word; its bit is picked at the store
    };
    auto stage_load = [&](const Geo& g, int j0, Raw& rw) {
        const int iy = j0 / PT, ix = j0 % PT;
        const int y = g.y0 - 3 + iy, x = g.x0 - 3 + ix;
        const bool in = y >= 0 && y < g.H && x >= 0 && x < g.W;
        // every load is issued, from an address inside the cloth (a node
        // outside reads its nearest cloth node and counts as zero), so that
        // all of a helper's loads are in flight together
        const int yc = min(max(y, 0), g.H - 1), xc = min(max(x, 0), g.W - 1);
        const float* p0 = g.src + (int64_t)yc * g.rs + (STEP ? col_pos(xc) : xc);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float r = __ldg(p0 + c * g.cs);
            rw.v[c] = in ? r : 0.f;
        }
        rw.pin = 0;
        if constexpr (STEP) {
            const int oy = iy - 3, ox = ix - 3;
            const uint32_t pw = __ldg(g.pin + (int64_t)yc * g.pin_wpr + (xc >> 5));
            if (in && oy >= 0 && oy < R && ox >= 0 && ox < WO) rw.pin = pw;
        }
    };
    auto stage_store = [&](const Geo& g, int buf, int j0, const Raw& rw) {
        const int iy = j0 / PT, ix = j0 % PT;
        float v[8];
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = sIns[c] * rw.v[c];
        v[6] = v[7] = 0.f;
        if constexpr (SPLIT) {   // v = hi + lo, both BF16
            float lo[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) lo[c] = v[c] - __bfloat162float(__float2bfloat16_rn(v[c]));
            sIn(buf, 0)[j0] = pack8(v);
            sIn(buf, 1)[j0] = pack8(lo);
        } else {
            sIn(buf)[j0] = pack8(v);
        }
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
    auto stage = [&](const Geo& g, int tile, int buf) {   // the whole region at once
        if (STEP && tid == 0) {
            sD[buf] = A.desc[g.cloth];
            sTile[buf] = A.tiles[tile];
        }
        for (int j0 = tid; j0 < N0; j0 += NWORK) {
            Raw rw;
            stage_load(g, j0, rw);
            stage_store(g, buf, j0, rw);
        }
    };
    constexpr int kHelpParts = (N0 + NHELP - 1) / NHELP;   // input nodes per helper

    // The edge terms of a tile, from its staged input (workers, once per
    // tile, spread over all of them): for each cell-region node on an edge
    // of the cloth and each of the 96 output columns, the 5 taps of that
    // edge's correction along the edge, and for a node on an x edge that is
    // also on a y edge the add-back of the term both corrections removed.
    // Slots: x = 0 by cell row, x = W-1 by cell row, y = 0 by cell column,
    // y = H-1 by cell column.
    auto edge_prep = [&](const Geo& g, const uint4* in, float* corr, int t, int nthr) {
        const int kGroups = nthr / kNC;   // node groups: thread t -> (column n, group gi)
        if (t >= kGroups * kNC) return;
        const int n = t % kNC, gi = t / kNC;
        if (n >= 59 && n < 64) return;   // padding columns: never read
        const int rxE = g.W - g.x0, ryN = g.H - g.y0;   // cell column of x = W-1, cell row of y = H-1
        // the edges present (bit ed), as a mask: no array indexed by the
        // edge loop's counter, which would live in local memory
        const uint32_t has = (uint32_t)(g.x0 == 0) | (uint32_t)(rxE >= 0 && rxE < WO + 2) << 1 |
                             (uint32_t)(g.y0 == 0) << 2 | (uint32_t)(ryN >= 0 && ryN < R + 2) << 3;
        if (has == 0) return;   // an interior tile: no edge terms
        // the three input slots of column n: u (n < 64) or v
        auto z3 = [&](int row, float (&z)[3]) {
            const uint4 r = in[row];
            if (n < 64) { z[0] = bf_lo(r.x); z[1] = bf_hi(r.x); z[2] = bf_lo(r.y); }
            else { z[0] = bf_hi(r.y); z[1] = bf_lo(r.z); z[2] = bf_hi(r.z); }
            if constexpr (SPLIT) {   // + the low part: the FP32 value the MMAs see
                const uint4 l = in[row + N0BUF];
                if (n < 64) { z[0] += bf_lo(l.x); z[1] += bf_hi(l.x); z[2] += bf_lo(l.y); }
                else { z[0] += bf_hi(l.y); z[1] += bf_lo(l.z); z[2] += bf_hi(l.z); }
            }
        };
        const float* gKD = SPLIT ? reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(A.wpack) + kOffKD2)
                                 : reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(A.wpack) + kBc) + kKE + kKC;
#pragma unroll 1
        for (int ed = 0; ed < 4; ++ed) {
            if (!((has >> ed) & 1u)) continue;
            const int base = ed < 2 ? ed * (R + 2) : 2 * (R + 2) + (ed - 2) * (WO + 2);   // the edge's first slot
            // the rounding defect of a tap is added by the first edge (in the
            // order x = 0, x = W-1, y = 0, y = H-1) whose column or row holds
            // it: x = W-1 leaves its column to x = 0 on a one-column cloth,
            // y = H-1 its row to y = 0 on a one-row cloth, and a y edge leaves
            // the centre tap to an x edge its node is on (decided per node)
            const bool none = (ed == 1 && g.W == 1) || (ed == 3 && g.H == 1);
            float k[15], kdc[3], kc[2][3];
#pragma unroll
            for (int j = 0; j < 15; ++j) {
                const float d = none ? 0.f : __ldg(gKD + ((ed >> 1) * 5 + j / 3) * 3 * kNC + (j % 3) * kNC + n);
                k[j] = __ldg(gKE + (ed * 5 + j / 3) * 3 * kNC + (j % 3) * kNC + n);
                if (j / 3 == 2) kdc[j % 3] = d;
                else k[j] += d;
            }
#pragma unroll
            for (int yb = 0; yb < 2; ++yb)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) kc[yb][ch] = ed < 2 ? __ldg(gKC + (2 * yb + ed) * 3 * kNC + ch * kNC + n) : 0.f;
            const int len = ed < 2 ? R + 2 : WO + 2;
#pragma unroll 1
            for (int i = gi; i < len; i += kGroups) {
                const int ry2 = ed < 2 ? i : (ed == 2 ? 1 : ryN), rx2 = ed < 2 ? (ed == 0 ? 1 : rxE) : i;
                const int y = g.y0 - 1 + ry2, x = g.x0 - 1 + rx2;
                if (y < 0 || y >= g.H || x < 0 || x >= g.W) continue;   // not a node of the cloth
                const int j2 = ry2 * PT + rx2;
                const bool ctr = !(ed >= 2 && (x == 0 || x == g.W - 1));
                float acc = 0.f;
#pragma unroll
                for (int s5 = 0; s5 < 5; ++s5) {   // x edges: taps along y; y edges: along x
                    float z[3];
                    z3(j2 + (ed < 2 ? s5 * PT + 2 : 2 * PT + s5), z);
                    float k0 = k[3 * s5], k1 = k[3 * s5 + 1], k2 = k[3 * s5 + 2];
                    if (s5 == 2 && ctr) {
                        k0 += kdc[0]; k1 += kdc[1]; k2 += kdc[2];
                    }
                    acc = fmaf(k0, z[0], fmaf(k1, z[1], fmaf(k2, z[2], acc)));
                }
                if (ed < 2 && (y == 0 || y == g.H - 1)) {   // corners (ay, ax): k4 = 2 (ay / 2) + ax / 2
                    float z[3];
                    z3(j2 + 2 * PT + 2, z);
#pragma unroll
                    for (int yb = 0; yb < 2; ++yb)
                        if (yb ? y == g.H - 1 : y == 0)
                            acc = fmaf(kc[yb][0], z[0], fmaf(kc[yb][1], z[1], fmaf(kc[yb][2], z[2], acc)));
                }
                corr[(base + i) * kCorrW + n] = acc;
            }
        }
    };

    // 3. epilogue of chunk c2 (accumulator b): the edge corrections;
    // s = tanh(t) and xi . s of the channel group [8 cg, +8) into the BF16
    // A operand of the N + D MMA (rows: the chunk's 128 positions); q, the
    // WL partial sums, into sQ (zero outside the cloth: WL's zero padding)
    auto epilogue = [&](const Geo& g, int c2, int b, const float* corr) {
        tc::fence_after();
        const int j2 = c2 * 128 + quarter * 32 + lane;
        const int ry2 = j2 / PT, rx2 = j2 % PT;
        const int y = g.y0 - 1 + ry2, x = g.x0 - 1 + rx2;
        const bool valid = j2 < N2 && rx2 < WO + 2 && y >= 0 && y < g.H && x >= 0 && x < g.W;
        const int oy = ry2 - 1, ox = rx2 - 1;
        const bool out_node = valid && oy >= 0 && oy < R && ox >= 0 && ox < WO;
        const uint32_t col = lane_base + (uint32_t)kNC * (uint32_t)b + 8u * (uint32_t)cg;
        float t[8], xi[8], q[8];
        tmem_ld8(col, t);
        tmem_ld8(col + 64, xi);
        tmem_ld8(col + 32, q);   // q_{8 cg} .. q_{8 cg + 7} (group 3: q_24..26 and padding)
        tc::tmem_wait_ld();
        if constexpr (SPLIT) {   // the accumulator is in registers: the issuer may refill it now
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(bar_read(b));
        }
        if (valid && (x == 0 || y == 0 || x == g.W - 1 || y == g.H - 1)) {
            auto add = [&](int slot) {
                const float4* c = reinterpret_cast<const float4*>(corr + slot * kCorrW + 8 * cg);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float4 a = c[j], e = c[8 + j], d = c[16 + j];
                    t[4 * j] += a.x; t[4 * j + 1] += a.y; t[4 * j + 2] += a.z; t[4 * j + 3] += a.w;
                    q[4 * j] += e.x; q[4 * j + 1] += e.y; q[4 * j + 2] += e.z; q[4 * j + 3] += e.w;
                    xi[4 * j] += d.x; xi[4 * j + 1] += d.y; xi[4 * j + 2] += d.z; xi[4 * j + 3] += d.w;
                }
            };
            if (x == 0) add(ry2);
            if (x == g.W - 1) add(R + 2 + ry2);
            if (y == 0) add(2 * (R + 2) + rx2);
            if (y == g.H - 1) add(2 * (R + 2) + WO + 2 + rx2);
        }
        if (j2 < N2 && rx2 < WO + 2) {
            float* qr = sQ + 8 * cg * NQ + ry2 * (WO + 2) + rx2;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < 3 || cg < 3) qr[k * NQ] = valid ? q[k] : 0.f;
        }
        if constexpr (SPLIT) {
            // s = tanh(t) in FP32 (the 1e-4 tolerance rules out tanh.approx)
            // and this channel group's share of N + D = WN s + WD (xi . s)
            float nd[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float sv = tanh_exp(t[c]), xs = xi[c] * sv;
#pragma unroll
                for (int co = 0; co < 3; ++co)
                    nd[co] = fmaf(sNDW[3 * kC + co * kC + 8 * cg + c], xs, fmaf(sNDW[co * kC + 8 * cg + c], sv, nd[co]));
            }
#pragma unroll
            for (int co = 0; co < 3; ++co) sND[(cg * 3 + co) * (C2 * 128) + j2] = nd[co];
        } else {
            // every row of the operand is written (rows that are no output
            // node give N + D nobody reads; their inputs are finite)
            float sv[8], xs[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                sv[c] = tc::tanh_approx(t[c]);
                xs[c] = xi[c] * sv[c];
            }
            uint4* a = reinterpret_cast<uint4*>(sm + oAnd + b * kAnd) + quarter * 32 + lane;
            a[cg * 128] = pack8(sv);
            a[(4 + cg) * 128] = pack8(xs);
            tc::fence_async_smem();   // the operand, for the tensor cores
        }
        tc::fence_before();
        (void)out_node;
    };

    // 4. per output node: L, N + D from tensor memory, a, and (step mode)
    // the update (workers).  Worker warp w takes cell-region row 4 (w / 4) +
    // w % 4 = the TMEM lane quarter w % 4 of chunk w / 4, so each thread
    // reads its own position's N + D.  Returns false if the N + D MMAs did
    // not finish in time.
    auto final_pass = [&](const Geo& g, int buf) {
        const float* sUb = sU + buf * kUFloats;
        const int cc = warp >> 2;
        const int j2 = cc * 128 + quarter * 32 + lane;   // ry2 = j2 / PT, rx2 = lane (PT = 32)
        const int oy = j2 / PT - 1, ox = j2 % PT - 1;
        float nd[4] = {0.f, 0.f, 0.f, 0.f};
        if constexpr (SPLIT) {   // the 4 channel groups' shares, in a fixed order
            if (j2 < N2) {
#pragma unroll
                for (int co = 0; co < 3; ++co) {
                    const float* p = sND + co * (C2 * 128) + j2;
                    nd[co] = ((p[0] + p[3 * C2 * 128]) + p[6 * C2 * 128]) + p[9 * C2 * 128];
                }
            }
        } else {
            const bool ok = tc::mbar_wait(bar_nd, ph_nd, kWaitLimit);
            ph_nd ^= 1u;
            tc::fence_after();
            uint32_t r[4];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                         : "r"(lane_base + kTmemND + (uint32_t)(kNDN * cc))
                         : "memory");
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 4; ++i) nd[i] = __uint_as_float(r[i]);
            tc::fence_before();
            if (!ok) return false;
        }
        const int o = oy * WO + ox, y = g.y0 + oy, x = g.x0 + ox;
        if (oy >= 0 && oy < R && ox >= 0 && ox < WO && y < g.H && x < g.W) {
            float acc[3];
#pragma unroll
            for (int co = 0; co < 3; ++co) {
                float L = sBL[co];
#pragma unroll
                for (int tap = 0; tap < 9; ++tap)
                    L += sQ[(tap * 3 + co) * NQ + (oy + tap / 3) * (WO + 2) + ox + tap % 3];
                acc[co] = sOut[co] * (L + nd[co]);
            }
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
        return true;
    };

    // ---- the pipeline.  Prologue: stage the first tile, issue its first two
    // chunks and compute its edge terms.
    static_assert(C2 >= 2, "two chunks in flight");
    int tile = skip((int)blockIdx.x);
    int buf = 0;
    int tn = n_tiles;
    if (tile < n_tiles) {
        const Geo g = geo(tile);
        tn = skip(tile + (int)gridDim.x);
        if (worker) {
            stage(g, tile, 0);
            tc::fence_async_smem();
        }
        __syncthreads();
        if (issuer) {
            issue_chunk(0, 0);
            issue_chunk(1, 0);
        }
        if (worker) edge_prep(g, sIn(0), sCorr(0), tid, NWORK);
        __syncthreads();
    }
    while (tile < n_tiles && !timed_out) {
        const bool has_next = tn < n_tiles;
        const int tnn = has_next ? skip(tn + (int)gridDim.x) : n_tiles;
        // the geometry each role needs: the workers this tile's (from shared
        // memory) and, after the chunks, the next one's for its edge terms;
        // the helpers the next one's from global memory
        Geo g{}, gn{};
        if (helper) {
            if (has_next) gn = geo(tn);
        } else if (worker) {
            g = geo_s(tile, buf);
        }
        bool ok = true;
        if (helper) {
            // 1. the next tile's input, descriptor and pinned flags while this
            // tile's chunks run, all of a helper's input nodes in flight at once
            if (has_next) {
                constexpr int kDescV = (int)(sizeof(ClothDesc) / sizeof(uint4));
                static_assert(sizeof(ClothDesc) % sizeof(uint4) == 0 && kDescV < NHELP, "descriptor copy");
                if (STEP && htid < kDescV)
                    reinterpret_cast<uint4*>(sD + (buf ^ 1))[htid] = reinterpret_cast<const uint4*>(A.desc + gn.cloth)[htid];
                if (STEP && htid == kDescV) sTile[buf ^ 1] = A.tiles[tn];
                constexpr int kBatch = kHelpParts;   // input nodes in flight per helper
#pragma unroll 1
                for (int k0 = 0; k0 < kHelpParts; k0 += kBatch) {
                    Raw rw[kBatch];
#pragma unroll
                    for (int k = 0; k < kBatch; ++k)
                        if (htid + (k0 + k) * NHELP < N0) stage_load(gn, htid + (k0 + k) * NHELP, rw[k]);
#pragma unroll
                    for (int k = 0; k < kBatch; ++k)
                        if (htid + (k0 + k) * NHELP < N0) stage_store(gn, buf ^ 1, htid + (k0 + k) * NHELP, rw[k]);
                }
                tc::fence_async_smem();   // the staged input, for the tensor cores
            }
        } else {
            // 2-3. the chunks of this tile, double-buffered in TMEM (chunk c+1
            // runs while the workers read chunk c).  No CTA barrier between
            // them: each worker warp reports its reads of an accumulator (and
            // its part of the N + D operand) on that accumulator's "free"
            // barrier; the issuer waits there, issues the chunk's N + D MMA and
            // then reuses the accumulator; after the last chunk's N + D it
            // commits to bar_nd, which the final pass waits for.  The FP32
            // form has no N + D MMA: the workers also arrive on the
            // accumulator's "read" barrier right after loading it, and the
            // issuer refills it from there.
            // BF16: unrolled, so the accumulator index and its barrier phases
            // are compile-time (no local-memory array); the FP32 form, with
            // more live registers, is faster rolled
#pragma unroll(SPLIT ? 1 : C2)
            for (int c2 = 0; c2 < C2; ++c2) {
                const int b = c2 & 1;
                if (worker) {
                    if (ok) ok = tc::mbar_wait(bar(b), (ph >> b) & 1u, kWaitLimit);
                    if (ok) {
                        epilogue(g, c2, b, sCorr(buf));   // FP32 form: arrives on bar_read(b) after its loads
                    } else if (SPLIT) {
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(bar_read(b));   // after a timeout: the issuer's wait ends
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(bar_free(b));   // also after a timeout: the issuer's wait ends
                }
                ph ^= 1u << b;
                if (issuer && ok) {
                    if constexpr (SPLIT) {
                        // no N + D MMA: the accumulator is refilled as soon as
                        // it is read, while the epilogue still runs (the free
                        // barrier has no waiter in this form)
                        ok = wait_read(b);
                        if (ok && c2 + 2 < C2) issue_chunk(c2 + 2, buf);
                    } else {
                        ok = wait_free(b);
                        if (ok) {
                            issue_nd(c2);
                            if (c2 + 2 < C2) issue_chunk(c2 + 2, buf);
                            if (c2 == C2 - 1) tc::mma_commit(bar_nd);
                        }
                    }
                }
            }
        }

        // the next tile's first two chunks run during this tile's final pass
        if (__syncthreads_or(!ok)) { timed_out = true; break; }
        if (issuer && has_next) {   // the accumulators were freed by the last two chunks
            issue_chunk(0, buf ^ 1);
            issue_chunk(1, buf ^ 1);
        }
        if (worker) {
            if (!final_pass(g, buf)) ok = false;
            if (has_next) {   // this tile's epilogues are done; the helpers staged the next tile
                gn = geo_s(tn, buf ^ 1);
                edge_prep(gn, sIn(buf ^ 1), sCorr(buf ^ 1), tid, NWORK);
            }
        }
        if (__syncthreads_or(!ok)) { timed_out = true; break; }
        tile = tn;
        tn = tnn;
        buf ^= 1;
    }

    // ---- tear-down: the issuer commits once more, so bar_drain completes
    // when every MMA it issued is done (after a timeout some may still be
    // in flight); tensor memory is freed after that (bounded) wait
    if (timed_out && tid == 0 && A.status) atomicOr(A.status, kStatusTimeout);
    if (issuer) tc::mma_commit(bar_drain);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        if (!tc::mbar_wait(bar_drain, 0, kWaitLimit) && lane == 0 && A.status) atomicOr(A.status, kStatusTimeout);
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// Composite tap (cy, cx) of output column n and input slot e in FP32: the
// sum over a + b = c of the layer products, in one fixed order (the B
// operand and the rounding defects both come from it).
__device__ float composite_tap(const float* __restrict__ w, int n, int e, int cy, int cx)
{
    float v = 0.f;
    for (int ay = 0; ay < 3; ++ay)
        for (int ax = 0; ax < 3; ++ax) {
            const int by = cy - ay, bx = cx - ax;
            if (by >= 0 && by < 3 && bx >= 0 && bx < 3) v += trunk_composite(w, n, e, 3 * ay + ax, 3 * by + bx);
        }
    return v;
}

// The composite operands from the FP32 blob, one thread per value (the
// algebra is trunk_composite).
__global__ void pack_tc_kernel(const float* __restrict__ w, uint8_t* __restrict__ out)
{
    constexpr int nB = kPairs * 2 * kNC * 8;
    constexpr int nFirst = nB + kKE + kKC + kKD + kNDK * kNDN;   // up to the three-term split's tables
    const int r0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (r0 >= nFirst + nB + kKD) return;
    auto tap = [](int y, int x) { return 3 * y + x; };
    if (r0 >= nFirst + nB) {   // KD2: the composite tap less Bhi + Blo, in KD's layout
        const int q3 = r0 - nFirst - nB;
        const int n = q3 % kNC, ch = (q3 / kNC) % 3, s5 = (q3 / (3 * kNC)) % 5, dir = q3 / (15 * kNC);
        float d = 0.f;
        if (n < 59 || n >= 64) {
            const float v = composite_tap(w, n, n < 64 ? ch : 3 + ch, dir == 0 ? s5 : 2, dir == 0 ? 2 : s5);
            const float hi = __bfloat162float(__float2bfloat16_rn(v));
            d = v - (hi + __bfloat162float(__float2bfloat16_rn(v - hi)));
        }
        reinterpret_cast<float*>(out + kOffKD2)[q3] = d;
        return;
    }
    if (r0 >= nFirst) {   // Blo: BF16(B - Bhi), in B's layout
        const int r = r0 - nFirst;
        const int e = r % 8, n = (r / 8) % kNC, kh = (r / (8 * kNC)) % 2, p = r / (16 * kNC);
        const int c = 2 * p + kh, cy = c / 5, cx = c % 5;
        float v = 0.f;
        const bool u_col = n < 59 && e < 3, v_col = n >= 64 && e >= 3 && e < 6;
        if (c < 25 && (u_col || v_col)) v = composite_tap(w, n, e, cy, cx);
        const float hi = __bfloat162float(__float2bfloat16_rn(v));
        reinterpret_cast<__nv_bfloat16*>(out + kOffBlo)[r] = __float2bfloat16_rn(v - hi);
        return;
    }
    const int r = r0;
    if (r >= nB + kKE + kKC + kKD) {   // B of N + D: [k / 8][n][k % 8]
        const int e2 = r - (nB + kKE + kKC + kKD);
        const int e = e2 % 8, n = (e2 / 8) % kNDN, k = (e2 / (8 * kNDN)) * 8 + e;
        float v = 0.f;
        if (n < 3) v = k < kC ? w[kOffWN + n * kC + k] : w[kOffWD + n * kC + (k - kC)];
        reinterpret_cast<__nv_bfloat16*>(out + kOffBnd)[e2] = __float2bfloat16_rn(v);
        return;
    }
    if (r < nB) {   // B: tap pair p, the pair's first (kh 0) or second tap, column n, input slot e
        const int e = r % 8, n = (r / 8) % kNC, kh = (r / (8 * kNC)) % 2, p = r / (16 * kNC);
        const int c = 2 * p + kh, cy = c / 5, cx = c % 5;
        float v = 0.f;
        const bool u_col = n < 59 && e < 3, v_col = n >= 64 && e >= 3 && e < 6;
        if (c < 25 && (u_col || v_col)) v = composite_tap(w, n, e, cy, cx);
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        reinterpret_cast<__nv_bfloat16*>(out)[r] = h;
        return;
    }
    float* fo = reinterpret_cast<float*>(out + kBc);
    if (r >= nB + kKE + kKC) {   // KD: direction dir, tap s, channel ch, column n
        const int q3 = r - nB - kKE - kKC;
        const int n = q3 % kNC, ch = (q3 / kNC) % 3, s5 = (q3 / (3 * kNC)) % 5, dir = q3 / (15 * kNC);
        float d = 0.f;
        if (n < 59 || n >= 64) {
            const float v = composite_tap(w, n, n < 64 ? ch : 3 + ch, dir == 0 ? s5 : 2, dir == 0 ? 2 : s5);
            d = v - __bfloat162float(__float2bfloat16_rn(v));
        }
        fo[kKE + kKC + q3] = d;
        return;
    }
    const int q = r - nB;
    if (q < kKE) {   // edge ed, tap s along the edge, channel ch, column n
        const int n = q % kNC, ch = (q / kNC) % 3, s = (q / (3 * kNC)) % 5, ed = q / (15 * kNC);
        float v = 0.f;
        if (n < 59 || n >= 64) {
            const int i = n < 64 ? ch : 3 + ch;
            // x = 0: the layer-1 column x - 1 (a_x = 0) is outside and only
            // b_x = 2 reaches back into the cloth; x = W - 1: a_x = 2, b_x = 0;
            // y = 0: a_y = 0, b_y = 2; y = H - 1: a_y = 2, b_y = 0
            for (int k = 0; k < 3; ++k) {
                const int m = s - k;
                if (m < 0 || m > 2) continue;
                int a, b;
                if (ed == 0) { a = tap(k, 0); b = tap(m, 2); }
                else if (ed == 1) { a = tap(k, 2); b = tap(m, 0); }
                else if (ed == 2) { a = tap(0, k); b = tap(2, m); }
                else { a = tap(2, k); b = tap(0, m); }
                v -= trunk_composite(w, n, i, a, b);
            }
        }
        fo[q] = v;
        return;
    }
    const int q2 = q - kKE;   // corner k4 = (ay / 2) * 2 + ax / 2, channel ch, column n
    const int n = q2 % kNC, ch = (q2 / kNC) % 3, k4 = q2 / (3 * kNC);
    float v = 0.f;
    if (n < 59 || n >= 64) {
        const int ay = (k4 >> 1) * 2, ax = (k4 & 1) * 2;
        v = trunk_composite(w, n, n < 64 ? ch : 3 + ch, tap(ay, ax), tap(2 - ay, 2 - ax));
    }
    fo[kKE + q2] = v;
}

}  // namespace

int net_tc_pack_bytes() { return kPack; }
int net_tc_edge_offset() { return kBc; }
int net_tc_tile_cols() { return WO; }
// BF16 tile shapes v = 0, 1, 2: 4, 3 or 2 chunks (14, 10 or 6 output rows);
// the FP32 three-term shapes k = 0, 1: 3 or 2 chunks (10 or 6 rows; 4 chunks
// of the split operands do not fit in shared memory)
int net_tc_variants() { return 3; }
int net_tc_variant_rows(int v) { return 4 * (4 - v) - 2; }
int net_tc_split_variants() { return 2; }
int net_tc_split_rows(int k) { return 4 * (3 - k) - 2; }

namespace {
template <bool STEP, int C2, bool SPLIT>
cudaError_t set_smem()
{
    return cudaFuncSetAttribute(net_tc_kernel<STEP, C2, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TcShape<C2, SPLIT>::kSmem);
}
template <int C2, bool SPLIT>
void launch_step(const TcArgs& a, int grid, cudaStream_t s)
{
    net_tc_kernel<true, C2, SPLIT><<<grid, NTH, TcShape<C2, SPLIT>::kSmem, s>>>(a);
}
}  // namespace

cudaError_t net_tc_init()
{
    cudaError_t e = set_smem<true, 4, false>();
    if (e == cudaSuccess) e = set_smem<true, 3, false>();
    if (e == cudaSuccess) e = set_smem<true, 2, false>();
    if (e == cudaSuccess) e = set_smem<true, 3, true>();
    if (e == cudaSuccess) e = set_smem<true, 2, true>();
    if (e == cudaSuccess) e = set_smem<false, 4, false>();
    return e;
}

cudaError_t launch_pack_bf16(const float* w, void* wpack, cudaStream_t s)
{
    constexpr int n = 2 * kPairs * 2 * kNC * 8 + kKE + kKC + 2 * kKD + kNDK * kNDN;
    pack_tc_kernel<<<(n + 127) / 128, 128, 0, s>>>(w, static_cast<uint8_t*>(wpack));
    return cudaGetLastError();
}

cudaError_t launch_net_tc_step(int variant, bool split, const void* wpack, const float* w, const ClothDesc* desc,
                               const int4* tiles, int n_tiles, const float* src, float* dst, const uint32_t* pinmask,
                               int32_t* status, int grid, cudaStream_t s, const int32_t* mode)
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
    if (split) {
        if (variant == 1) launch_step<2, true>(a, grid, s);
        else launch_step<3, true>(a, grid, s);
    } else if (variant == 1) launch_step<3, false>(a, grid, s);
    else if (variant == 2) launch_step<2, false>(a, grid, s);
    else launch_step<4, false>(a, grid, s);
    return cudaGetLastError();
}

cudaError_t launch_net_tc_forward(const void* wpack, const float* w, const float* z, float* out, int N, int H, int W,
                                  int32_t* status, int grid, cudaStream_t s)
{
    using S = TcShape<4, false>;
    TcArgs a{};
    a.wpack = static_cast<const uint4*>(wpack);
    a.w = w;
    a.status = status;
    a.z = z;
    a.a = out;
    a.N = N; a.H = H; a.W = W;
    a.tiles_y = (H + S::R - 1) / S::R;
    a.tiles_x = (W + WO - 1) / WO;
    const int n_tiles = N * a.tiles_y * a.tiles_x;
    net_tc_kernel<false, 4, false><<<grid < n_tiles ? grid : n_tiles, NTH, S::kSmem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace cloth
