// CNN cell (Sec. 3.2, Eq. 6-7) in FP32 on CUDA cores: forward with saved
// activations and the hand-written backward (the cell and training path;
// the FP32 network step is the fused kernel of net_comp.cu).
//
// Layer by layer, NCHW FP32 activations, every 3x3 convolution a tiled
// kernel: a block of 128 threads computes a 32 x 8 tile of nodes for all
// output channels (each thread 2 nodes, rows ty and ty + 4), with the input
// tile plus its 1-node halo and the weights staged in shared memory.  Weight
// gradients are per-block partial sums over a fixed assignment of tiles,
// reduced in a fixed order, so results are bitwise reproducible.
#include "net_internal.cuh"

namespace cloth {
namespace {

constexpr int TW = 32, TH = 8, NT = 128;

// ----------------------------------------------------------------- views
// Cell input, field f of image n: f = 0 -> in_scale[0:3] u, f = 1 ->
// in_scale[3:6] v.  Image index img = 2 n + f.
struct InZ {
    NetSrc src;
    const float* w;
    int H, W;
    __device__ float operator()(int img, int c, int y, int x) const
    {
        const int n = img >> 1, f = img & 1;
        const float sc = w[kOffIns + 3 * f + c];
        return sc * src.z[(((int64_t)n * 6 + 3 * f + c) * H + y) * W + x];
    }
};

// Plain NCHW tensor: image i at p + (i * img_mul + img_add) * img_stride.
struct View {
    const float* p;
    int64_t img_stride, HW;
    int W, img_mul, img_add;
    __device__ float operator()(int i, int c, int y, int x) const
    {
        return p[(int64_t)(i * img_mul + img_add) * img_stride + c * HW + (int64_t)y * W + x];
    }
};

struct ProdView {   // elementwise product of two views (xi . s)
    View a, b;
    __device__ float operator()(int i, int c, int y, int x) const { return a(i, c, y, x) * b(i, c, y, x); }
};

struct Ones {
    __device__ float operator()(int, int, int, int) const { return 1.f; }
};

// Field f of the scaled cell input of image n: in_scale[3f + c] z[n][3f + c].
struct ZView {
    const float* z;
    const float* w;
    int64_t HW;
    int W, f;
    __device__ float operator()(int n, int c, int y, int x) const
    {
        return w[kOffIns + 3 * f + c] * z[((int64_t)n * 6 + 3 * f + c) * HW + (int64_t)y * W + x];
    }
};

struct OutView {
    float* p;
    int64_t img_stride, HW;
    int W;
    __device__ void operator()(int i, int c, int y, int x, float v) const
    {
        p[(int64_t)i * img_stride + c * HW + (int64_t)y * W + x] = v;
    }
};

// d z output of field f = img & 1 into channels 3 f .. 3 f + 2, times in_scale.
struct OutGz {
    float* gz;
    const float* w;
    int H, W;
    __device__ void operator()(int img, int c, int y, int x, float v) const
    {
        const int n = img >> 1, f = img & 1;
        gz[(((int64_t)n * 6 + 3 * f + c) * H + y) * W + x] = w[kOffIns + 3 * f + c] * v;
    }
};

// ----------------------------------------------------------------- weights
// W(o, i, tap) of the convolution computed: o = output, i = input channel.
struct WtW1 {   // phi1 / xi1 = W1 (*) [zu; 0] / [0; zv]: field f uses W1[:, 3f:3f+3]
    const float* w;
    __device__ float operator()(int img, int o, int i, int tap) const
    {
        return w[kOffW1 + (o * 6 + 3 * (img & 1) + i) * 9 + tap];
    }
};
struct WtW2 {
    const float* w;
    __device__ float operator()(int, int o, int i, int tap) const { return w[kOffW2 + (o * kC + i) * 9 + tap]; }
};
// Transposed convolutions (adjoint wrt the input): swap the channel roles
// and flip the taps.
struct WtW2T {
    const float* w;
    __device__ float operator()(int, int o, int i, int tap) const { return w[kOffW2 + (i * kC + o) * 9 + (8 - tap)]; }
};
struct WtW1T {
    const float* w;
    __device__ float operator()(int img, int o, int i, int tap) const
    {
        return w[kOffW1 + (i * 6 + 3 * (img & 1) + o) * 9 + (8 - tap)];
    }
};

// ----------------------------------------------------------------- staging
// Element e (0 <= e < count) of a tile: value get(e) stored by put(e, value).
// Each thread issues kBatch loads before it stores any of them, so a batch
// costs one memory latency instead of kBatch (the source is reached through
// a generic pointer, so the compiler would not move the loads above the
// shared-memory stores by itself).
constexpr int kBatch = 8;
template <class Get, class Put>
__device__ __forceinline__ void stage_tile(int count, int tid, int nthreads, Get get, Put put)
{
    for (int e0 = tid; e0 < count; e0 += kBatch * nthreads) {
        float v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int e = e0 + k * nthreads;
            v[k] = e < count ? get(e) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int e = e0 + k * nthreads;
            if (e < count) put(e, v[k]);
        }
    }
}

// ----------------------------------------------------------------- conv
// out(img, o, y, x) = sum_{i, ky, kx} W(o, i, ky, kx) in(img, i, y+ky-1, x+kx-1)
// with zero outside [0, H) x [0, W).  Grid: (tiles_x, tiles_y, images).
template <int CIN, int COUT, class In, class Wt, class Out>
__global__ void __launch_bounds__(NT) conv3x3_kernel(In in, Wt wt, Out out, int H, int W)
{
    constexpr int COUTP = (COUT + 3) / 4 * 4;
    extern __shared__ float4 smem4[];
    float* s_w = reinterpret_cast<float*>(smem4);          // [9][CIN][COUTP]
    float* s_in = s_w + 9 * CIN * COUTP;                   // [CIN][TH+2][TW+2]
    const int img = blockIdx.z, x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int tid = threadIdx.x;
    stage_tile(9 * CIN * COUTP, tid, NT, [&](int e) {
        const int tap = e / (CIN * COUTP), rem = e % (CIN * COUTP), i = rem / COUTP, o = rem % COUTP;
        return o < COUT ? wt(img, o, i, tap) : 0.f;
    }, [&](int e, float v) { s_w[e] = v; });
    stage_tile(CIN * (TH + 2) * (TW + 2), tid, NT, [&](int e) {
        const int i = e / ((TH + 2) * (TW + 2)), rem = e % ((TH + 2) * (TW + 2));
        const int y = y0 + rem / (TW + 2) - 1, x = x0 + rem % (TW + 2) - 1;
        return (y >= 0 && y < H && x >= 0 && x < W) ? in(img, i, y, x) : 0.f;
    }, [&](int e, float v) { s_in[e] = v; });
    __syncthreads();
    const int tx = tid & 31, ty = tid >> 5;
    float acc0[COUTP], acc1[COUTP];
#pragma unroll
    for (int o = 0; o < COUTP; ++o) acc0[o] = acc1[o] = 0.f;
    for (int i = 0; i < CIN; ++i) {
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const float* si = s_in + (i * (TH + 2) + ty + ky) * (TW + 2) + tx + kx;
                const float a0 = si[0], a1 = si[4 * (TW + 2)];
                const float4* w4 = reinterpret_cast<const float4*>(s_w + ((ky * 3 + kx) * CIN + i) * COUTP);
#pragma unroll
                for (int q = 0; q < COUTP / 4; ++q) {
                    const float4 w = w4[q];
                    acc0[4 * q + 0] = fmaf(w.x, a0, acc0[4 * q + 0]); acc1[4 * q + 0] = fmaf(w.x, a1, acc1[4 * q + 0]);
                    acc0[4 * q + 1] = fmaf(w.y, a0, acc0[4 * q + 1]); acc1[4 * q + 1] = fmaf(w.y, a1, acc1[4 * q + 1]);
                    acc0[4 * q + 2] = fmaf(w.z, a0, acc0[4 * q + 2]); acc1[4 * q + 2] = fmaf(w.z, a1, acc1[4 * q + 2]);
                    acc0[4 * q + 3] = fmaf(w.w, a0, acc0[4 * q + 3]); acc1[4 * q + 3] = fmaf(w.w, a1, acc1[4 * q + 3]);
                }
            }
    }
    const int x = x0 + tx;
    if (x < W) {
        if (y0 + ty < H)
#pragma unroll
            for (int o = 0; o < COUT; ++o) out(img, o, y0 + ty, x, acc0[o]);
        if (y0 + ty + 4 < H)
#pragma unroll
            for (int o = 0; o < COUT; ++o) out(img, o, y0 + ty + 4, x, acc1[o]);
    }
}

template <int CIN, int COUT>
constexpr int conv_smem() { return (9 * CIN * ((COUT + 3) / 4 * 4) + CIN * (TH + 2) * (TW + 2)) * 4; }

template <int CIN, int COUT, class In, class Wt, class Out>
cudaError_t conv3x3(In in, Wt wt, Out out, int H, int W, int images, cudaStream_t s)
{
    if (images <= 0 || H <= 0 || W <= 0) return cudaSuccess;
    dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, images);
    conv3x3_kernel<CIN, COUT, In, Wt, Out><<<grid, NT, conv_smem<CIN, COUT>(), s>>>(in, wt, out, H, W);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- branches
// Eq. 7 on the trunk output t2 = (phi, xi): L = WL (*) phi + bL,
// s = tanh(P phi), N = WN s, D = WD (xi . s), a = out_scale (L + N + D).
constexpr int kBranchSmem = (3 * kC * 9 + kC * kC + 6 * kC + 8 + kC * (TH + 2) * (TW + 2)) * 4;

__global__ void __launch_bounds__(NT) branch_fwd_kernel(const float* __restrict__ w, const float* __restrict__ t2,
                                                        float* __restrict__ s_out, float* __restrict__ a, int H, int W)
{
    extern __shared__ float4 smem4[];
    float* sWL = reinterpret_cast<float*>(smem4);     // [3][32][9]
    float* sP = sWL + 3 * kC * 9;                     // [32][32]
    float* sWN = sP + kC * kC;                        // [3][32]
    float* sWD = sWN + 3 * kC;                        // [3][32]
    float* sB = sWD + 3 * kC;                         // bL[3], out_scale[3]
    float* sPhi = sB + 8;                             // [32][TH+2][TW+2]
    const int n = blockIdx.z, x0 = blockIdx.x * TW, y0 = blockIdx.y * TH, tid = threadIdx.x;
    const int64_t HW = (int64_t)H * W;
    stage_tile(3 * kC * 9, tid, NT, [&](int e) { return w[kOffWL + e]; }, [&](int e, float v) { sWL[e] = v; });
    stage_tile(kC * kC, tid, NT, [&](int e) { return w[kOffP + e]; }, [&](int e, float v) { sP[e] = v; });
    for (int e = tid; e < 3 * kC; e += NT) { sWN[e] = w[kOffWN + e]; sWD[e] = w[kOffWD + e]; }
    if (tid < 3) { sB[tid] = w[kOffBL + tid]; sB[3 + tid] = w[kOffOuts + tid]; }
    const float* phi = t2 + (int64_t)n * 2 * kC * HW;
    const float* xi = phi + kC * HW;
    stage_tile(kC * (TH + 2) * (TW + 2), tid, NT, [&](int e) {
        const int i = e / ((TH + 2) * (TW + 2)), rem = e % ((TH + 2) * (TW + 2));
        const int y = y0 + rem / (TW + 2) - 1, x = x0 + rem % (TW + 2) - 1;
        return (y >= 0 && y < H && x >= 0 && x < W) ? phi[i * HW + (int64_t)y * W + x] : 0.f;
    }, [&](int e, float v) { sPhi[e] = v; });
    __syncthreads();
    // each thread's two nodes (rows ly and ly + 4) in one pass, so every
    // weight read from shared memory serves both (each node's sums keep
    // their order)
    const int tx = tid & 31, x = x0 + tx, ly = tid >> 5;
    const int ya = y0 + ly, yb = ya + 4;
    if (x >= W || ya >= H) return;   // yb > ya: both out
    const bool hb = yb < H;
    const int64_t pa = (int64_t)ya * W + x, pb = hb ? (int64_t)yb * W + x : pa;
    float La[3] = {sB[0], sB[1], sB[2]}, Lb[3] = {sB[0], sB[1], sB[2]};
    for (int i = 0; i < kC; ++i)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const float va = sPhi[(i * (TH + 2) + ly + ky) * (TW + 2) + tx + kx];
                const float vb = sPhi[(i * (TH + 2) + ly + 4 + ky) * (TW + 2) + tx + kx];
#pragma unroll
                for (int o = 0; o < 3; ++o) {
                    const float wl = sWL[(o * kC + i) * 9 + ky * 3 + kx];
                    La[o] = fmaf(wl, va, La[o]);
                    Lb[o] = fmaf(wl, vb, Lb[o]);
                }
            }
    float pca[kC], pcb[kC];
#pragma unroll
    for (int i = 0; i < kC; ++i) {
        pca[i] = sPhi[(i * (TH + 2) + ly + 1) * (TW + 2) + tx + 1];
        pcb[i] = sPhi[(i * (TH + 2) + ly + 5) * (TW + 2) + tx + 1];
    }
    float Na[3] = {0.f, 0.f, 0.f}, Da[3] = {0.f, 0.f, 0.f}, Nb[3] = {0.f, 0.f, 0.f}, Db[3] = {0.f, 0.f, 0.f};
    for (int c = 0; c < kC; ++c) {
        float ta = 0.f, tb = 0.f;
        const float4* pr = reinterpret_cast<const float4*>(sP + c * kC);
#pragma unroll
        for (int q = 0; q < kC / 4; ++q) {
            const float4 pw = pr[q];
            ta = fmaf(pw.x, pca[4 * q], fmaf(pw.y, pca[4 * q + 1], fmaf(pw.z, pca[4 * q + 2], fmaf(pw.w, pca[4 * q + 3], ta))));
            tb = fmaf(pw.x, pcb[4 * q], fmaf(pw.y, pcb[4 * q + 1], fmaf(pw.z, pcb[4 * q + 2], fmaf(pw.w, pcb[4 * q + 3], tb))));
        }
        const float sa = tanhf(ta), sb = tanhf(tb);
        const float xsa = xi[c * HW + pa] * sa, xsb = xi[c * HW + pb] * sb;
        if (s_out) {
            s_out[((int64_t)n * kC + c) * HW + pa] = sa;
            if (hb) s_out[((int64_t)n * kC + c) * HW + pb] = sb;
        }
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            Na[o] = fmaf(sWN[o * kC + c], sa, Na[o]);
            Da[o] = fmaf(sWD[o * kC + c], xsa, Da[o]);
            Nb[o] = fmaf(sWN[o * kC + c], sb, Nb[o]);
            Db[o] = fmaf(sWD[o * kC + c], xsb, Db[o]);
        }
    }
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        a[((int64_t)n * 3 + o) * HW + pa] = sB[3 + o] * (La[o] + Na[o] + Da[o]);
        if (hb) a[((int64_t)n * 3 + o) * HW + pb] = sB[3 + o] * (Lb[o] + Nb[o] + Db[o]);
    }
}

// Backward through Eq. 7 at every node: from d a to d y = out_scale d a,
// d xi, d t = d s (1 - s^2) and d phi = P^T d t + WL^T (*) d y.
__global__ void __launch_bounds__(NT) branch_bwd_kernel(const float* __restrict__ w, const float* __restrict__ ga,
                                                        float* __restrict__ saved, int H, int W)
{
    extern __shared__ float4 smem4[];
    float* sWL = reinterpret_cast<float*>(smem4);     // [3][32][9]
    float* sP = sWL + 3 * kC * 9;                     // [32][32]
    float* sWN = sP + kC * kC;
    float* sWD = sWN + 3 * kC;
    float* sB = sWD + 3 * kC;                         // out_scale[3]
    float* sGy = sB + 8;                              // [3][TH+2][TW+2]
    const int n = blockIdx.z, N = gridDim.z, x0 = blockIdx.x * TW, y0 = blockIdx.y * TH, tid = threadIdx.x;
    const int64_t HW = (int64_t)H * W, NHW = (int64_t)N * HW;
    stage_tile(3 * kC * 9, tid, NT, [&](int e) { return w[kOffWL + e]; }, [&](int e, float v) { sWL[e] = v; });
    stage_tile(kC * kC, tid, NT, [&](int e) { return w[kOffP + e]; }, [&](int e, float v) { sP[e] = v; });
    for (int e = tid; e < 3 * kC; e += NT) { sWN[e] = w[kOffWN + e]; sWD[e] = w[kOffWD + e]; }
    if (tid < 3) sB[tid] = w[kOffOuts + tid];
    __syncthreads();
    for (int e = tid; e < 3 * (TH + 2) * (TW + 2); e += NT) {
        const int o = e / ((TH + 2) * (TW + 2)), rem = e % ((TH + 2) * (TW + 2));
        const int y = y0 + rem / (TW + 2) - 1, x = x0 + rem % (TW + 2) - 1;
        sGy[e] = (y >= 0 && y < H && x >= 0 && x < W) ? sB[o] * ga[((int64_t)n * 3 + o) * HW + (int64_t)y * W + x] : 0.f;
    }
    __syncthreads();
    const float* xi = saved + kSavT2 * NHW + ((int64_t)n * 2 + 1) * kC * HW;
    const float* sv = saved + kSavS * NHW + (int64_t)n * kC * HW;
    float* gphi = saved + kSavG2 * NHW + (int64_t)n * 2 * kC * HW;
    float* gxi = gphi + kC * HW;
    float* gt = saved + kSavGT * NHW + (int64_t)n * kC * HW;
    float* gy = saved + kSavGY * NHW + (int64_t)n * 3 * HW;
    // each thread's two nodes (rows ly and ly + 4) in one pass, so every
    // weight read from shared memory serves both (each node's sums keep
    // their order)
    const int tx = tid & 31, x = x0 + tx, ly = tid >> 5;
    const int ya = y0 + ly, yb = ya + 4;
    if (x >= W || ya >= H) return;   // yb > ya: both out
    const bool hb = yb < H;
    const int64_t pa = (int64_t)ya * W + x, pb = hb ? (int64_t)yb * W + x : pa;
    float g0[3], g1[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        g0[o] = sGy[(o * (TH + 2) + ly + 1) * (TW + 2) + tx + 1];
        g1[o] = sGy[(o * (TH + 2) + ly + 5) * (TW + 2) + tx + 1];
        gy[o * HW + pa] = g0[o];
        if (hb) gy[o * HW + pb] = g1[o];
    }
    float gtla[kC], gtlb[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) {
        const float sa = sv[c * HW + pa], xa = xi[c * HW + pa];
        const float sb = sv[c * HW + pb], xb = xi[c * HW + pb];
        float gxsa = 0.f, gsa = 0.f, gxsb = 0.f, gsb = 0.f;
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            gxsa = fmaf(sWD[o * kC + c], g0[o], gxsa);
            gsa = fmaf(sWN[o * kC + c], g0[o], gsa);
            gxsb = fmaf(sWD[o * kC + c], g1[o], gxsb);
            gsb = fmaf(sWN[o * kC + c], g1[o], gsb);
        }
        gsa = fmaf(gxsa, xa, gsa);
        gsb = fmaf(gxsb, xb, gsb);
        gtla[c] = gsa * (1.f - sa * sa);
        gtlb[c] = gsb * (1.f - sb * sb);
        gxi[c * HW + pa] = gxsa * sa;
        gt[c * HW + pa] = gtla[c];
        if (hb) {
            gxi[c * HW + pb] = gxsb * sb;
            gt[c * HW + pb] = gtlb[c];
        }
    }
    for (int i = 0; i < kC; ++i) {
        float acca = 0.f, accb = 0.f;
#pragma unroll
        for (int c = 0; c < kC; ++c) {
            const float pw = sP[c * kC + i];
            acca = fmaf(pw, gtla[c], acca);
            accb = fmaf(pw, gtlb[c], accb);
        }
        // WL^T (*) d y: d phi_i(p) += sum_o,ky,kx WL[o][i][ky][kx] d y_o(p - (ky-1, kx-1))
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                for (int o = 0; o < 3; ++o) {
                    const float wl = sWL[(o * kC + i) * 9 + ky * 3 + kx];
                    acca = fmaf(wl, sGy[(o * (TH + 2) + ly + 2 - ky) * (TW + 2) + tx + 2 - kx], acca);
                    accb = fmaf(wl, sGy[(o * (TH + 2) + ly + 6 - ky) * (TW + 2) + tx + 2 - kx], accb);
                }
        gphi[i * HW + pa] = acca;
        if (hb) gphi[i * HW + pb] = accb;
    }
}

// ----------------------------------------------------------------- wgrad
// Partial weight gradients: for the tiles t = blockIdx.x, + gridDim.x, ...
// (tile = 32 x 8 nodes of image i), out[(a * BSTRIDE + b) * TAPS + tap] +=
// sum_pixels A(i, a, y, x) B(i, b, y + dy, x + dx) with B zero outside the
// image.  Thread (pg, ab, b) owns a in [ab*ABLK, ab*ABLK+ABLK), one b, and the
// tile rows pg, pg + PG, ...: shapes with few (a, b) pairs take several row
// groups per block, whose sums are added in a fixed order at the end, so the
// partials stay bitwise reproducible.
template <int CA, int CB, int TAPS, int ABLK>
struct WgradShape {
    static constexpr int NG = (CA / ABLK) * CB;                       // threads of one row group
    static constexpr int PG = NG >= 256 ? 1 : (256 / NG < TH ? 256 / NG : TH);
    static constexpr int NTH = NG * PG < 32 ? 32 : NG * PG;
    static constexpr int HB = TAPS == 9 ? 1 : 0;                      // halo of the B tile
    static constexpr int kTile = CA * TH * TW + CB * ((TH + 2 * HB) * (TW + 2 * HB) + 1);
    static constexpr int kRed = PG > 1 ? PG * CA * CB * TAPS : 0;
    static constexpr int kSmem = (kTile > kRed ? kTile : kRed) * 4;
};

template <int CA, int CB, int TAPS, int ABLK, class AV, class BV>
__global__ void wgrad_kernel(AV A, BV B, float* __restrict__ part, int out_off, int bstride, int H, int W, int n_img)
{
    using S = WgradShape<CA, CB, TAPS, ABLK>;
    constexpr int HB = S::HB, PG = S::PG;
    extern __shared__ float4 smem4[];
    float* sA = reinterpret_cast<float*>(smem4);          // [CA][TH][TW]
    float* sB = sA + CA * TH * TW;                          // [CB][TH+2HB][TW+2HB] (+1 pad)
    constexpr int BW = TW + 2 * HB, BH = TH + 2 * HB, BPL = BH * BW + 1;
    const int tid = threadIdx.x;
    const int pg = tid / S::NG, r = tid % S::NG, ab = r / CB, b = r % CB;
    const bool active = pg < PG && ab < CA / ABLK;
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    const int n_tiles = tiles_x * tiles_y * n_img;
    float acc[ABLK][TAPS];
#pragma unroll
    for (int j = 0; j < ABLK; ++j)
#pragma unroll
        for (int t = 0; t < TAPS; ++t) acc[j][t] = 0.f;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int i = tile / (tiles_x * tiles_y), rem = tile % (tiles_x * tiles_y);
        const int y0 = (rem / tiles_x) * TH, x0 = (rem % tiles_x) * TW;
        __syncthreads();
        stage_tile(CA * TH * TW, tid, blockDim.x, [&](int e) {
            const int a = e / (TH * TW), r2 = e % (TH * TW), y = y0 + r2 / TW, x = x0 + r2 % TW;
            return (y < H && x < W) ? A(i, a, y, x) : 0.f;
        }, [&](int e, float v) { sA[e] = v; });
        stage_tile(CB * BH * BW, tid, blockDim.x, [&](int e) {
            const int bb = e / (BH * BW), r2 = e % (BH * BW);
            const int y = y0 + r2 / BW - HB, x = x0 + r2 % BW - HB;
            return (y >= 0 && y < H && x >= 0 && x < W) ? B(i, bb, y, x) : 0.f;
        }, [&](int e, float v) { sB[(e / (BH * BW)) * BPL + e % (BH * BW)] = v; });
        __syncthreads();
        if (active) {
            for (int py = pg; py < TH; py += PG) {
                // 3 x 3 taps: a window of B's columns px .. px + 2 slides along
                // the row, one new column (3 loads) per node
                float win[3][3];
                if constexpr (TAPS == 9) {
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy) {
                        win[dy][1] = sB[b * BPL + (py + dy) * BW + 0];
                        win[dy][2] = sB[b * BPL + (py + dy) * BW + 1];
                    }
                }
                for (int px = 0; px < TW; ++px) {
                    float av[ABLK];
#pragma unroll
                    for (int j = 0; j < ABLK; ++j) av[j] = sA[((ab * ABLK + j) * TH + py) * TW + px];
                    if constexpr (TAPS == 9) {
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy) {
                            win[dy][0] = win[dy][1];
                            win[dy][1] = win[dy][2];
                            win[dy][2] = sB[b * BPL + (py + dy) * BW + px + 2];
                        }
                    }
#pragma unroll
                    for (int t = 0; t < TAPS; ++t) {
                        const int dy = TAPS == 9 ? t / 3 : 0, dx = TAPS == 9 ? t % 3 : 0;
                        const float bv = TAPS == 9 ? win[dy][dx] : sB[b * BPL + py * BW + px];
#pragma unroll
                        for (int j = 0; j < ABLK; ++j) acc[j][t] = fmaf(av[j], bv, acc[j][t]);
                    }
                }
            }
        }
    }
    float* out = part + (int64_t)blockIdx.x * kParams + out_off;
    if constexpr (PG == 1) {
        if (active) {
#pragma unroll
            for (int j = 0; j < ABLK; ++j)
#pragma unroll
                for (int t = 0; t < TAPS; ++t) out[((ab * ABLK + j) * bstride + b) * TAPS + t] = acc[j][t];
        }
    } else {
        // the row groups' sums, added in the order pg = 0, 1, ...
        float* red = reinterpret_cast<float*>(smem4);   // [PG][CA][CB][TAPS]
        __syncthreads();
        if (active) {
#pragma unroll
            for (int j = 0; j < ABLK; ++j)
#pragma unroll
                for (int t = 0; t < TAPS; ++t) red[((pg * CA + ab * ABLK + j) * CB + b) * TAPS + t] = acc[j][t];
        }
        __syncthreads();
        if (active && pg == 0) {
#pragma unroll
            for (int j = 0; j < ABLK; ++j)
#pragma unroll
                for (int t = 0; t < TAPS; ++t) {
                    float sum = 0.f;
                    for (int q = 0; q < PG; ++q) sum += red[((q * CA + ab * ABLK + j) * CB + b) * TAPS + t];
                    out[((ab * ABLK + j) * bstride + b) * TAPS + t] = sum;
                }
        }
    }
}

template <int CA, int CB, int TAPS, int ABLK, class AV, class BV>
cudaError_t wgrad(AV A, BV B, float* part, int out_off, int bstride, int H, int W, int n_img, cudaStream_t s)
{
    using S = WgradShape<CA, CB, TAPS, ABLK>;
    wgrad_kernel<CA, CB, TAPS, ABLK, AV, BV><<<kWgradBlocks, S::NTH, S::kSmem, s>>>(A, B, part, out_off, bstride, H, W,
                                                                                  n_img);
    return cudaGetLastError();
}

// gw[j] += sum over blocks g (in order) of part[g][j]
__global__ void reduce_partials_kernel(const float* __restrict__ part, float* __restrict__ gw)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kParams) return;
    float s = 0.f;
    for (int g = 0; g < kWgradBlocks; ++g) s += part[(int64_t)g * kParams + j];
    gw[j] += s;
}

}  // namespace

cudaError_t net_simt_init()
{
    cudaError_t e;
#define SET_SMEM(kern, bytes)                                                                   \
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) \
        return e;
    SET_SMEM((conv3x3_kernel<3, kC, InZ, WtW1, OutView>), (conv_smem<3, kC>()));
    SET_SMEM((conv3x3_kernel<kC, kC, View, WtW2, OutView>), (conv_smem<kC, kC>()));
    SET_SMEM((conv3x3_kernel<kC, kC, View, WtW2T, OutView>), (conv_smem<kC, kC>()));
    SET_SMEM((conv3x3_kernel<kC, 3, View, WtW1T, OutGz>), (conv_smem<kC, 3>()));
    SET_SMEM(branch_fwd_kernel, kBranchSmem);
    SET_SMEM(branch_bwd_kernel, kBranchSmem);
    SET_SMEM((wgrad_kernel<kC, kC, 9, 4, View, View>), (WgradShape<kC, kC, 9, 4>::kSmem));
    SET_SMEM((wgrad_kernel<kC, kC, 1, 4, View, View>), (WgradShape<kC, kC, 1, 4>::kSmem));
#undef SET_SMEM
    return conv32_tc_init();
}

cudaError_t launch_net_forward_simt(const NetFwdArgs& f, cudaStream_t s)
{
    const int H = f.H, W = f.W, N = f.N;
    const int64_t HW = (int64_t)H * W;
    cudaError_t e;
    // Eq. 6: phi1 = W1 (*) [zu; 0], xi1 = W1 (*) [0; zv] (images 2n + field)
    e = conv3x3<3, kC>(InZ{f.src, f.w, H, W}, WtW1{f.w}, OutView{f.t1, kC * HW, HW, W}, H, W, 2 * N, s);
    if (e != cudaSuccess) return e;
    // phi = W2 (*) phi1, xi = W2 (*) xi1: on the tensor cores where a status
    // word can report a timed-out wait
    if (f.status)
        e = launch_conv32_tc(f.t1, f.t2, f.w, false, 2 * N, H, W, f.status, s);
    else
        e = conv3x3<kC, kC>(View{f.t1, kC * HW, HW, W, 1, 0}, WtW2{f.w}, OutView{f.t2, kC * HW, HW, W}, H, W, 2 * N, s);
    if (e != cudaSuccess) return e;
    // Eq. 7
    dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, N);
    branch_fwd_kernel<<<grid, NT, kBranchSmem, s>>>(f.w, f.t2, f.s, f.a, H, W);
    return cudaGetLastError();
}

cudaError_t launch_net_backward_simt(const float* w, const float* z, float* saved, const float* ga, float* gz,
                                     float* part, float* gw, int N, int H, int W, int32_t* status, cudaStream_t s)
{
    const int64_t HW = (int64_t)H * W, NHW = (int64_t)N * HW;
    float* T1 = saved + kSavT1 * NHW;
    float* T2 = saved + kSavT2 * NHW;
    float* Sv = saved + kSavS * NHW;
    float* G2 = saved + kSavG2 * NHW;
    float* GT = saved + kSavGT * NHW;
    float* GY = saved + kSavGY * NHW;
    cudaError_t e;
    dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, N);
    branch_bwd_kernel<<<grid, NT, kBranchSmem, s>>>(w, ga, saved, H, W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const View gy{GY, 3 * HW, HW, W, 1, 0};
    const View phi{T2, 2 * kC * HW, HW, W, 1, 0};          // image n -> T2[n][0]
    const View xi{T2 + kC * HW, 2 * kC * HW, HW, W, 1, 0};  // image n -> T2[n][1]
    const View sv{Sv, kC * HW, HW, W, 1, 0};
    const View gt{GT, kC * HW, HW, W, 1, 0};
    // weight gradients of Eq. 7: WL, bL, P, WN, WD
    if ((e = wgrad<3, kC, 9, 3>(gy, phi, part, kOffWL, kC, H, W, N, s)) != cudaSuccess) return e;
    if ((e = wgrad<3, 1, 1, 3>(gy, Ones{}, part, kOffBL, 1, H, W, N, s)) != cudaSuccess) return e;
    if ((e = wgrad<kC, kC, 1, 4>(gt, phi, part, kOffP, kC, H, W, N, s)) != cudaSuccess) return e;
    if ((e = wgrad<3, kC, 1, 3>(gy, sv, part, kOffWN, kC, H, W, N, s)) != cudaSuccess) return e;
    if ((e = wgrad<3, kC, 1, 3>(gy, ProdView{xi, sv}, part, kOffWD, kC, H, W, N, s)) != cudaSuccess) return e;
    // W2: d phi1 = W2^T (*) d phi (into the T2 region, now free), d W2
    float* G1 = T2;
    if ((e = wgrad<kC, kC, 9, 4>(View{G2, kC * HW, HW, W, 1, 0}, View{T1, kC * HW, HW, W, 1, 0}, part, kOffW2, kC, H, W,
                                 2 * N, s)) != cudaSuccess)
        return e;
    e = status ? launch_conv32_tc(G2, G1, w, true, 2 * N, H, W, status, s)
               : conv3x3<kC, kC>(View{G2, kC * HW, HW, W, 1, 0}, WtW2T{w}, OutView{G1, kC * HW, HW, W}, H, W, 2 * N, s);
    if (e != cudaSuccess) return e;
    // W1: per field, d W1[:, 3f:3f+3] from d phi1 / d xi1 and the scaled input
    for (int f = 0; f < 2; ++f) {
        if ((e = wgrad<kC, 3, 9, 4>(View{G1, kC * HW, HW, W, 2, f}, ZView{z, w, HW, W, f}, part, kOffW1 + 27 * f, 6, H, W,
                                    N, s)) != cudaSuccess)
            return e;
    }
    reduce_partials_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(part, gw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (gz)
        return conv3x3<kC, 3>(View{G1, kC * HW, HW, W, 1, 0}, WtW1T{w}, OutGz{gz, w, H, W}, H, W, 2 * N, s);
    return cudaSuccess;
}

}  // namespace cloth
