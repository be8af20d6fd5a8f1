// The network step (Fig. 2) with the CNN cell (Sec. 3.2, Eq. 6-7) in FP32
// on the CUDA cores, fused into one kernel.
//
// The trunk W2 (*) (W1 (*) z) is linear and bias-free and its output phi
// enters Eq. 7 only through P and WL, so per node the kernel evaluates one
// 5x5 composite convolution of the scaled input z: t = P C (*) u, the 27
// partial sums q_tap,co = WL[co][:][tap] C (*) u and xi = C (*) v, with
// C_c = sum_{a+b=c} W2_a W1_b — about 6,800 multiply-adds per node instead
// of the layered 22,240.  On the cloth's outermost ring the layers' zero
// padding is restored by the same edge and corner terms as the tensor-core
// step (FP32 tables packed with it), so every node gets the layered result.
//
// One block of 16 (TC + 2) threads per tile of 14 x TC output nodes,
// looping over the tiles; TC is 14 by default (256 threads, two blocks per
// SM), and 6 and 30 are the other tile shapes the launch tuner can pick.
// Per tile:
//   0. stage the 20 x (TC + 6) input region (scaled z, and the raw u, v of
//      the 16 x (TC + 2) cell region for the update), zero outside the cloth;
//   1. the composite convolution over the 16 x 16 cell region: a thread
//      takes four cell positions 4 rows apart and one of eight column groups
//      (t and xi channels [4 g, +4), q values [4 g, +4) below 27),
//      accumulates the 12 columns of the 4 positions in paired FP32 (f32x2)
//      FMAs with the weights read from shared memory (the same address for
//      the whole warp, each load feeding the 4 positions), adds the edge
//      terms, stores q and its channels' share of N + D = WN s + WD (xi . s),
//      s = tanh(t);
//   2. per output node: L = bL + sum_tap q_tap at the tap's neighbour, the
//      eight shares of N + D added in a fixed order, a = out_scale (L + N +
//      D), then v <- C(v + dt (a + f_p / m)), u <- u + dt v, sphere contact,
//      store.
#include "net_internal.cuh"

namespace cloth {
namespace {

constexpr int kGroups = 8, kGW = 12;       // column groups; weights per (group, tap, channel)
constexpr int kPos = 4;                    // cell positions per item, 4 rows apart
constexpr int kWF = kGroups * 25 * 3 * kGW;

// Tile shape 14 x TCOL and what follows from it.
template <int TCOL>
struct Shape {
    static constexpr int TR = 14, TC = TCOL;               // output tile
    static constexpr int CR = TR + 2, CC = TC + 2;         // cell region, origin (y0 - 1, x0 - 1)
    static constexpr int IR = TR + 6, IC = TC + 6;         // input region, origin (y0 - 3, x0 - 3)
    static constexpr int NCELL = CR * CC, NIN = IR * IC, NOUT = TR * TC;
    static constexpr int NTHR = 16 * CC;                   // two items of four positions per thread
    static constexpr int kQuads = NCELL / kPos;            // 4 CC
    static constexpr int kMinBlocks = TC <= 6 ? 3 : (TC <= 14 ? 2 : 1);
    // shared memory (bytes)
    static constexpr int oW = 0;                                  // composite weights [g][tap][ch][12]
    static constexpr int oZ = oW + kWF * 4;                       // scaled z: [NIN] float4 u0 u1 u2 v0, then [NIN] float2 v1 v2
    static constexpr int oRaw = oZ + NIN * 24;                    // raw u, v [6][NCELL]
    static constexpr int oQ = oRaw + 6 * NCELL * 4;               // q [27][NCELL]
    static constexpr int oND = oQ + 27 * NCELL * 4;               // N + D shares [g][NOUT][3]
    static constexpr int oPar = oND + kGroups * NOUT * 3 * 4;     // WND[32][8], bL[3], outs[3], ins[6]
    static constexpr int oDesc = oPar + (256 + 16) * 4;
    static constexpr int oPin = oDesc + (int)sizeof(ClothDesc);
    static constexpr int kSmem = oPin + (NOUT + 15) / 16 * 16;
    static_assert(kGroups * kQuads == 2 * NTHR && kQuads % 32 == 0, "two items of four positions per thread, one group per warp");
    static_assert(NOUT <= NTHR, "one output node per thread in the final pass");
    static_assert(kQuads == 4 * CC && CR == 4 * kPos, "the rows cy0 + 4 p of the quads cover the cell region once");
    static_assert(oZ % 16 == 0 && oRaw % 16 == 0 && oPar % 16 == 0 && oDesc % 16 == 0, "alignment");
    static_assert(kMinBlocks * (kSmem + 1024) <= 233472, "resident blocks per SM");
};
// the tile widths the launch tuner chooses among (index = variant)
constexpr int kVariants = 3;
constexpr int kVariantCols[kVariants] = {14, 6, 30};

struct CompArgs {
    const float* w;        // FP32 blob
    const float4* wf;      // composite weights, kWF floats
    const float* ke;       // edge terms [4][5][3][96], then corner terms [4][3][96]
    const ClothDesc* desc;
    const int4* tiles;     // (cloth, y0, x0, -)
    int n_tiles;
    const float* src;
    float* dst;
    const uint32_t* pinmask;
    const int32_t* mode;   // if set, only cloths in network mode are stepped
    int32_t* status;
};

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 F2(float a) { return make_float2(a, a); }

template <int TCOL>
__global__ void __launch_bounds__(Shape<TCOL>::NTHR, Shape<TCOL>::kMinBlocks) net_comp_kernel(CompArgs A)
{
    using S = Shape<TCOL>;
    constexpr int TR = S::TR, TC = S::TC, CR = S::CR, CC = S::CC, IC = S::IC;
    constexpr int NCELL = S::NCELL, NIN = S::NIN, NOUT = S::NOUT, NTHR = S::NTHR, kQuads = S::kQuads;
    constexpr int oW = S::oW, oZ = S::oZ, oRaw = S::oRaw, oQ = S::oQ, oND = S::oND, oPar = S::oPar;
    constexpr int oDesc = S::oDesc, oPin = S::oPin;
    extern __shared__ __align__(16) uint8_t sm[];
    const int tid = threadIdx.x;
    const float4* sW = reinterpret_cast<const float4*>(sm + oW);
    float4* sZa = reinterpret_cast<float4*>(sm + oZ);            // u0 u1 u2 v0 per input node
    float2* sZb = reinterpret_cast<float2*>(sm + oZ + NIN * 16);  // v1 v2
    float* sRaw = reinterpret_cast<float*>(sm + oRaw);
    float* sQ = reinterpret_cast<float*>(sm + oQ);
    float* sND = reinterpret_cast<float*>(sm + oND);
    float* sPar = reinterpret_cast<float*>(sm + oPar);
    const float4* sWND = reinterpret_cast<const float4*>(sm + oPar);   // [c][2]: WN0..2 WD0, WD1 WD2 0 0
    float* sBL = sPar + 256;
    float* sOut = sBL + 3;
    float* sIns = sOut + 3;
    ClothDesc* sD = reinterpret_cast<ClothDesc*>(sm + oDesc);
    uint8_t* sPin = sm + oPin;

    for (int e = tid; e < kWF / 4; e += NTHR) reinterpret_cast<float4*>(sm + oW)[e] = A.wf[e];
    for (int e = tid; e < 32 * 8; e += NTHR) {
        const int c = e >> 3, j = e & 7;
        sPar[e] = j < 3 ? A.w[kOffWN + j * kC + c] : (j < 6 ? A.w[kOffWD + (j - 3) * kC + c] : 0.f);
    }
    if (tid < 3) {
        sBL[tid] = A.w[kOffBL + tid];
        sOut[tid] = A.w[kOffOuts + tid];
    }
    if (tid < 6) sIns[tid] = A.w[kOffIns + tid];
    __syncthreads();

    for (int tile = blockIdx.x; tile < A.n_tiles; tile += gridDim.x) {
        const int4 tt = A.tiles[tile];
        if (A.mode && A.mode[tt.x] != kModeNet) continue;   // the same for the whole block
        if (tid == 0) *sD = A.desc[tt.x];
        const int y0 = tt.y, x0 = tt.z;
        const int H = A.desc[tt.x].rows, W = A.desc[tt.x].cols;

        // 0. the input region
        {
            const ClothDesc& D = A.desc[tt.x];
            const float* src = A.src + D.plane_off;
            const uint32_t* pins = A.pinmask + D.pin_off;
            for (int j = tid; j < NIN; j += NTHR) {
                const int iy = j / IC, ix = j % IC, y = y0 - 3 + iy, x = x0 - 3 + ix;
                float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                const bool in = y >= 0 && y < H && x >= 0 && x < W;
                if (in) {
                    const float* p = src + (int64_t)y * D.pitch + col_pos(x);
#pragma unroll
                    for (int c = 0; c < 6; ++c) v[c] = __ldg(p + c * D.plane_stride);
                }
                sZa[j] = make_float4(sIns[0] * v[0], sIns[1] * v[1], sIns[2] * v[2], sIns[3] * v[3]);
                sZb[j] = make_float2(sIns[4] * v[4], sIns[5] * v[5]);
                const int cy = iy - 2, cx = ix - 2;
                if (cy >= 0 && cy < CR && cx >= 0 && cx < CC) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) sRaw[c * NCELL + cy * CC + cx] = v[c];
                }
                const int oy = iy - 3, ox = ix - 3;
                if (oy >= 0 && oy < TR && ox >= 0 && ox < TC)
                    sPin[oy * TC + ox] = in ? (uint8_t)((__ldg(pins + (int64_t)y * D.pin_wpr + (x >> 5)) >> (x & 31)) & 1u) : 0;
            }
        }
        __syncthreads();

        // 1. the composite convolution, two items per thread: column group g
        // (the same for a whole warp) and cell positions p0 + 4 k CC, k < 4
#pragma unroll 1
        for (int r = 0; r < 2; ++r) {
            const int item = r * NTHR + tid, g = item / kQuads, p0 = item % kQuads;
            const int cy0 = p0 / CC, cx = p0 % CC;
            float2 acc[kPos][6];   // t pairs 0-1, xi pairs 2-3, q pairs 4-5
#pragma unroll
            for (int p = 0; p < kPos; ++p)
#pragma unroll
                for (int k = 0; k < 6; ++k) acc[p][k] = F2(0.f);
#pragma unroll 1
            for (int ty = 0; ty < 5; ++ty) {
#pragma unroll 1
                for (int tx = 0; tx < 5; ++tx) {
                    const int i0 = (cy0 + ty) * IC + cx + tx;
                    float zu[kPos][3], zv[kPos][3];
#pragma unroll
                    for (int p = 0; p < kPos; ++p) {
                        const float4 a = sZa[i0 + 4 * p * IC];
                        const float2 b = sZb[i0 + 4 * p * IC];
                        zu[p][0] = a.x; zu[p][1] = a.y; zu[p][2] = a.z;
                        zv[p][0] = a.w; zv[p][1] = b.x; zv[p][2] = b.y;
                    }
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const float4* wp = sW + ((g * 25 + ty * 5 + tx) * 3 + ch) * 3;
                        const float4 wt = wp[0], wx = wp[1], wq = wp[2];
#pragma unroll
                        for (int p = 0; p < kPos; ++p) {
                            const float2 u = F2(zu[p][ch]), vv = F2(zv[p][ch]);
                            acc[p][0] = fma2(make_float2(wt.x, wt.y), u, acc[p][0]);
                            acc[p][1] = fma2(make_float2(wt.z, wt.w), u, acc[p][1]);
                            acc[p][2] = fma2(make_float2(wx.x, wx.y), vv, acc[p][2]);
                            acc[p][3] = fma2(make_float2(wx.z, wx.w), vv, acc[p][3]);
                            acc[p][4] = fma2(make_float2(wq.x, wq.y), u, acc[p][4]);
                            acc[p][5] = fma2(make_float2(wq.z, wq.w), u, acc[p][5]);
                        }
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < kPos; ++p) {
                const int cy = cy0 + 4 * p, cell = cy * CC + cx;
                const int y = y0 - 1 + cy, x = x0 - 1 + cx;
                const bool valid = y >= 0 && y < H && x >= 0 && x < W;
                float* col = reinterpret_cast<float*>(acc[p]);   // t [0, 4), xi [4, 8), q [8, 12)
                if (valid && (x == 0 || y == 0 || x == W - 1 || y == H - 1)) {
                    // the edge terms of this node's 12 columns: z at input (cy + 2 + dy, cx + 2 + dx)
                    const bool e[4] = {x == 0, x == W - 1, y == 0, y == H - 1};
                    auto add = [&](const float* K, int zi) {   // K = [3][96] of one tap
                        const float4 a = sZa[zi];
                        const float2 b = sZb[zi];
                        const float zu3[3] = {a.x, a.y, a.z}, zv3[3] = {a.w, b.x, b.y};
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) {
                            const float* k = K + ch * 96;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                col[j] = fmaf(__ldg(k + 4 * g + j), zu3[ch], col[j]);
                                col[4 + j] = fmaf(__ldg(k + 64 + 4 * g + j), zv3[ch], col[4 + j]);
                                if (4 * g + j < 27) col[8 + j] = fmaf(__ldg(k + 32 + 4 * g + j), zu3[ch], col[8 + j]);
                            }
                        }
                    };
#pragma unroll 1
                    for (int ed = 0; ed < 4; ++ed) {
                        if (!e[ed]) continue;
#pragma unroll 1
                        for (int s5 = 0; s5 < 5; ++s5)
                            add(A.ke + (ed * 5 + s5) * 3 * 96, ed < 2 ? (cy + s5) * IC + cx + 2 : (cy + 2) * IC + cx + s5);
                    }
#pragma unroll 1
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const bool yo = (k4 >> 1) ? e[3] : e[2], xo = (k4 & 1) ? e[1] : e[0];
                        if (yo && xo) add(A.ke + 4 * 5 * 3 * 96 + k4 * 3 * 96, (cy + 2) * IC + cx + 2);
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (4 * g + j < 27) sQ[(4 * g + j) * NCELL + cell] = valid ? col[8 + j] : 0.f;
                const int oy = cy - 1, ox = cx - 1;
                if (valid && oy >= 0 && oy < TR && ox >= 0 && ox < TC) {
                    float nd0 = 0.f, nd1 = 0.f, nd2 = 0.f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float sv = tanhf(col[j]);
                        const float xs = col[4 + j] * sv;
                        const float4 w0 = sWND[2 * (4 * g + j)], w1 = sWND[2 * (4 * g + j) + 1];
                        nd0 = fmaf(w0.x, sv, fmaf(w0.w, xs, nd0));
                        nd1 = fmaf(w0.y, sv, fmaf(w1.x, xs, nd1));
                        nd2 = fmaf(w0.z, sv, fmaf(w1.y, xs, nd2));
                    }
                    float* o = sND + (g * NOUT + oy * TC + ox) * 3;
                    o[0] = nd0;
                    o[1] = nd1;
                    o[2] = nd2;
                }
            }
        }
        __syncthreads();

        // 2. per output node: L, a and the update
        if (tid < NOUT) {
            const int oy = tid / TC, ox = tid % TC, y = y0 + oy, x = x0 + ox;
            if (y < H && x < W) {
                const ClothDesc& D = *sD;
                float acc[3];
#pragma unroll
                for (int co = 0; co < 3; ++co) {
                    float L = sBL[co];
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) L += sQ[(tap * 3 + co) * NCELL + (oy + tap / 3) * CC + ox + tap % 3];
                    float nd = sND[tid * 3 + co];
#pragma unroll
                    for (int gg = 1; gg < kGroups; ++gg) nd += sND[(gg * NOUT + tid) * 3 + co];
                    acc[co] = sOut[co] * (L + nd);
                }
                auto U = [&](int ch, int cy, int cx) { return sRaw[ch * NCELL + cy * CC + cx]; };   // cell coordinates
                const int cy = oy + 1, cx = ox + 1;
                float u[3], v[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    u[c] = U(c, cy, cx);
                    v[c] = U(3 + c, cy, cx);
                }
                if (D.p_quarter != 0.f) {
                    const bool bE = x + 1 < W, bW = x > 0, bN = y + 1 < H, bS = y > 0;
                    float e[3], nn[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        e[c] = (bE ? U(c, cy, cx + 1) - u[c] + (c == 0 ? D.h : 0.f) : 0.f) -
                               (bW ? U(c, cy, cx - 1) - u[c] - (c == 0 ? D.h : 0.f) : 0.f);
                        nn[c] = (bN ? U(c, cy + 1, cx) - u[c] + (c == 1 ? D.h : 0.f) : 0.f) -
                                (bS ? U(c, cy - 1, cx) - u[c] - (c == 1 ? D.h : 0.f) : 0.f);
                    }
                    const float sc = D.p_quarter * D.inv_m;
                    acc[0] = fmaf(sc, e[1] * nn[2] - e[2] * nn[1], acc[0]);
                    acc[1] = fmaf(sc, e[2] * nn[0] - e[0] * nn[2], acc[1]);
                    acc[2] = fmaf(sc, e[0] * nn[1] - e[1] * nn[0], acc[2]);
                }
                const bool pinned = sPin[tid] != 0;
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
        __syncthreads();
    }
}

// The composite weights [g][tap][ch][12] from the FP32 blob, one thread per
// value: slots 0-3 t channel 4 g + e (input u_ch), 4-7 xi channel
// 4 g + e - 4 (input v_ch), 8-11 q value 4 g + e - 8 (input u_ch; none past
// 27).
__global__ void pack_comp_kernel(const float* __restrict__ w, float* __restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= kWF) return;
    const int e = r % kGW, ch = (r / kGW) % 3, c = (r / (3 * kGW)) % 25, g = r / (75 * kGW);
    int n = -1, i = ch;
    if (e < 4) n = 4 * g + e;
    else if (e < 8) { n = 64 + 4 * g + e - 4; i = 3 + ch; }
    else if (4 * g + e - 8 < 27) n = 32 + 4 * g + e - 8;
    float v = 0.f;
    if (n >= 0) {
        const int cy = c / 5, cx = c % 5;
        for (int ay = 0; ay < 3; ++ay)
            for (int ax = 0; ax < 3; ++ax) {
                const int by = cy - ay, bx = cx - ax;
                if (by >= 0 && by < 3 && bx >= 0 && bx < 3) v += trunk_composite(w, n, i, 3 * ay + ax, 3 * by + bx);
            }
    }
    out[r] = v;
}

}  // namespace

int net_comp_tile_rows() { return 14; }
int net_comp_variants() { return kVariants; }
int net_comp_variant_cols(int v) { return v >= 0 && v < kVariants ? kVariantCols[v] : 0; }
int net_comp_blocks_per_sm(int v)
{
    switch (v) {
    case 1: return Shape<6>::kMinBlocks;
    case 2: return Shape<30>::kMinBlocks;
    default: return Shape<14>::kMinBlocks;
    }
}
int net_comp_pack_floats() { return kWF; }

cudaError_t net_comp_init()
{
    cudaError_t e = cudaFuncSetAttribute(net_comp_kernel<14>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Shape<14>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(net_comp_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape<6>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(net_comp_kernel<30>, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape<30>::kSmem);
    return e;
}

cudaError_t launch_pack_comp(const float* w, float* out, cudaStream_t s)
{
    pack_comp_kernel<<<(kWF + 127) / 128, 128, 0, s>>>(w, out);
    return cudaGetLastError();
}

cudaError_t launch_net_comp_step(int variant, const float* w, const float* wf, const float* ke, const ClothDesc* desc,
                                 const int4* tiles, int n_tiles, const float* src, float* dst,
                                 const uint32_t* pinmask, int32_t* status, int grid, cudaStream_t s,
                                 const int32_t* mode)
{
    CompArgs a{};
    a.w = w;
    a.wf = reinterpret_cast<const float4*>(wf);
    a.ke = ke;
    a.desc = desc;
    a.tiles = tiles;
    a.n_tiles = n_tiles;
    a.src = src;
    a.dst = dst;
    a.pinmask = pinmask;
    a.mode = mode;
    a.status = status;
    switch (variant) {
    case 1: net_comp_kernel<6><<<grid, Shape<6>::NTHR, Shape<6>::kSmem, s>>>(a); break;
    case 2: net_comp_kernel<30><<<grid, Shape<30>::NTHR, Shape<30>::kSmem, s>>>(a); break;
    default: net_comp_kernel<14><<<grid, Shape<14>::NTHR, Shape<14>::kSmem, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace cloth
