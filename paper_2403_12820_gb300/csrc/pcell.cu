// The physics-embedded cell read literally (Sec. 3.2, Eq. 6-7, Fig. 1) and
// its network step (Fig. 2), for a batch of cloths in one launch.
//
// Eq. 6: the same 2D kernels act on every coordinate (isotropy), channel c
// being the frozen difference filter of one of the 12 stencil neighbours
// (the 3x3 ring and the dilation-2 cardinal taps): phi_c = x_j - x_i,
// xi_c = v_j - v_i, absent where the neighbour is outside the grid.
// Eq. 7 per coordinate: a = b_L + sum_c [w_L phi + w_N s + w_D xi s] with
// s = phi / sqrt(1 + alpha phi^2) (ISRU).
//
// Mapping: one block of 256 threads per 32 x 16 output tile; the tile and a
// 2-node halo of the six state planes are staged in shared memory (whole
// aligned groups of 4 columns, one float4 load each, all issued before any
// is stored); one thread per pair of nodes 8 rows apart, in f32x2 lanes.  phi is formed as l_c + (u_j - u_i) from the stored
// displacements u = x - X (l_c the lattice offset), which keeps the
// difference exact to the rounding of u.  Step mode adds the hard-encoded
// pressure (Eq. 3) and runs Eq. 5 with pins and sphere contact.
#include <type_traits>

#include "cloth_internal.cuh"

// Resident blocks of 256 threads per SM the register budget is sized for.
#ifndef CLOTH_PCELL_MINB
#define CLOTH_PCELL_MINB 4
#endif

namespace cloth {
namespace {

constexpr int TW = 32, TH = 16, HALO = 2;
constexpr int GX = 4;                                   // staged columns start 4 left of the tile
constexpr int SW = TW + 2 * GX, SH = TH + 2 * HALO;     // staged tile: 40 x 12
constexpr int NT = TW * TH / 2;                          // two nodes per thread
constexpr int kGroups = 6 * SH * (SW / 4);              // float4 loads per tile
constexpr int kLoadsPerThread = (kGroups + NT - 1) / NT;
static_assert(TW % 4 == 0, "tiles start on a column group");
constexpr int kPcellBlob = 40;

// channel offsets (row, column): E W N S NE NW SE SW E2 W2 N2 S2
__host__ __device__ constexpr int ch_dy(int c)
{
    return c == 2 || c == 4 || c == 5 ? 1 : (c == 3 || c == 6 || c == 7 ? -1 : (c == 10 ? 2 : (c == 11 ? -2 : 0)));
}
__host__ __device__ constexpr int ch_dx(int c)
{
    return c == 0 || c == 4 || c == 6 ? 1 : (c == 1 || c == 5 || c == 7 ? -1 : (c == 8 ? 2 : (c == 9 ? -2 : 0)));
}

struct PcellArgs {
    const ClothDesc* desc;
    const int4* tiles;     // (cloth, y0, x0, -)
    const float* w;        // w_L[12], w_N[12], w_D[12], b_L[3], alpha
    const float* src;
    float* dst;            // step mode: next state
    float* a_out;          // cell mode: acceleration, packed [node][3] (ABI order)
    const uint32_t* pinmask;
    int32_t* status;
};

using f2 = float2;
__device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, F2(-1.f), a); }

// Each thread computes nodes (y0 + ty, x) and (y0 + ty + TH / 2, x) as one
// pair of f32x2 lanes.
template <bool STEP>
__global__ void __launch_bounds__(NT, CLOTH_PCELL_MINB) pcell_kernel(PcellArgs A)
{
    __shared__ float sU[6][SH][SW];
    __shared__ float sW[kPcellBlob];
    // per channel (w_L, w_N, w_D, 0): one 16-byte shared load per channel
    __shared__ float4 sW4[12];
    const int4 t = A.tiles[blockIdx.x];
    const ClothDesc& D = A.desc[t.x];
    const int H = D.rows, W = D.cols;
    const int y0 = t.y, x0 = t.z;
    const int tid = threadIdx.x;
    if (tid < kPcellBlob) sW[tid] = A.w[tid];
    if (tid < 12) sW4[tid] = make_float4(A.w[tid], A.w[12 + tid], A.w[24 + tid], 0.f);
    const float* src = A.src + D.plane_off;
    const int pitch = D.pitch;
    const int64_t pstride = D.plane_stride;
    // group g: plane p, staged row r, columns x0 - 4 + 4 q .. +3 (in the
    // slots of col_slot); rows outside the grid and groups outside the pitch stay
    // zero (columns in the padding are zero in the state buffers)
    float4 ld[kLoadsPerThread];
#pragma unroll
    for (int i = 0; i < kLoadsPerThread; ++i) {
        const int g = tid + i * NT;
        const int p = g / (SH * (SW / 4)), r = (g / (SW / 4)) % SH, q = g % (SW / 4);
        const int y = y0 - HALO + r, xg = x0 - GX + 4 * q;
        ld[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (g < kGroups && y >= 0 && y < H && xg >= 0 && xg < pitch)
            ld[i] = __ldg(reinterpret_cast<const float4*>(src + p * pstride + (int64_t)y * pitch + xg));
    }
#pragma unroll
    for (int i = 0; i < kLoadsPerThread; ++i) {
        const int g = tid + i * NT;
        if (g >= kGroups) break;
        const int p = g / (SH * (SW / 4)), r = (g / (SW / 4)) % SH, q = g % (SW / 4);
        float* row = &sU[p][r][4 * q];
        const float tv[4] = {ld[i].x, ld[i].y, ld[i].z, ld[i].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) row[k] = tv[col_slot(k)];
    }
    __syncthreads();

    const int ty = tid / TW, tx = tid % TW;
    const int ya = y0 + ty, yb = ya + TH / 2, x = x0 + tx;
    if (ya >= H || x >= W) return;   // yb > ya: both out
    const bool hb = yb < H;          // second node exists
    const int sy = ty + HALO, sx = tx + GX;
    const float h = D.h;
    const f2 alpha = F2(sW[39]);
    auto U2 = [&](int p, int dy, int dx) { return make_float2(sU[p][sy + dy][sx + dx], sU[p][sy + TH / 2 + dy][sx + dx]); };
    // neighbour existence per node of the pair: rows -2 .. +2, columns -2 .. +2
    auto rowok = [&](int y, int dy) { return y + dy >= 0 && y + dy < H; };
    const bool c_m2 = x >= 2, c_m1 = x >= 1, c_p1 = x + 1 < W, c_p2 = x + 2 < W;
    f2 ui[3], vi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ui[k] = U2(k, 0, 0);
        vi[k] = U2(3 + k, 0, 0);
    }
    f2 acc[3] = {F2(sW[36]), F2(sW[37]), F2(sW[38])};
    // the 12 channels; a tile whose 2-node margin lies inside the grid has
    // every neighbour of both nodes (no existence masks)
    auto channels = [&](auto interior_tag) {
        constexpr bool kInterior = decltype(interior_tag)::value;
#pragma unroll
        for (int ch = 0; ch < 12; ++ch) {
            const int dy = ch_dy(ch), dx = ch_dx(ch);
            const float4 w4 = sW4[ch];
            f2 wl = F2(w4.x), wn = F2(w4.y), wd = F2(w4.z);
            if constexpr (!kInterior) {
                const bool cx = dx == 0 ? true : (dx == 1 ? c_p1 : (dx == -1 ? c_m1 : (dx == 2 ? c_p2 : c_m2)));
                const f2 m = make_float2(cx && rowok(ya, dy) ? 1.f : 0.f, cx && hb && rowok(yb, dy) ? 1.f : 0.f);
                wl = mul2(m, wl);
                wn = mul2(m, wn);
                wd = mul2(m, wd);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                // the lattice offset along coordinate k (none along z, nor
                // across the channel's direction: no add there)
                const int lk = k == 0 ? dx : (k == 1 ? dy : 0);
                const f2 du = sub2(U2(k, dy, dx), ui[k]);
                const f2 phi = lk == 0 ? du : add2(F2((float)lk * h), du);
                const f2 xi = sub2(U2(3 + k, dy, dx), vi[k]);
                // 1 + alpha phi^2 >= 1: never subnormal, the flushing form is exact here
                const f2 q = fma2(mul2(alpha, phi), phi, F2(1.f));
                const f2 s = mul2(phi, make_float2(rsqrt_ftz(q.x), rsqrt_ftz(q.y)));
                acc[k] = fma2(wl, phi, fma2(s, fma2(wd, xi, wn), acc[k]));
            }
        }
    };
    if (y0 >= HALO && y0 + TH + HALO <= H && x0 >= HALO && x0 + TW + HALO <= W)
        channels(std::true_type{});
    else
        channels(std::false_type{});
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        if (half == 1 && !hb) break;
        const int y = half ? yb : ya, yy = sy + half * (TH / 2);
        float a3[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) a3[k] = half ? acc[k].y : acc[k].x;
        if constexpr (!STEP) {
            float* o = A.a_out + (D.abi_off + (int64_t)y * W + x) * 3;
            o[0] = a3[0]; o[1] = a3[1]; o[2] = a3[2];
        } else {
            // pressure (Eq. 3): (p/4) (d'_E - d'_W) x (d'_N - d'_S) with absent
            // neighbours' terms dropped
            if (D.p_quarter != 0.f) {
                const bool bE = x + 1 < W, bW = x > 0, bN = y + 1 < H, bS = y > 0;
                float e[3], n[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float u0 = sU[k][yy][sx];
                    e[k] = (bE ? sU[k][yy][sx + 1] - u0 + (k == 0 ? h : 0.f) : 0.f) -
                           (bW ? sU[k][yy][sx - 1] - u0 - (k == 0 ? h : 0.f) : 0.f);
                    n[k] = (bN ? sU[k][yy + 1][sx] - u0 + (k == 1 ? h : 0.f) : 0.f) -
                           (bS ? sU[k][yy - 1][sx] - u0 - (k == 1 ? h : 0.f) : 0.f);
                }
                const float sc = D.p_quarter * D.inv_m;
                a3[0] = fmaf(sc, e[1] * n[2] - e[2] * n[1], a3[0]);
                a3[1] = fmaf(sc, e[2] * n[0] - e[0] * n[2], a3[1]);
                a3[2] = fmaf(sc, e[0] * n[1] - e[1] * n[0], a3[2]);
            }
            const bool pinned = (__ldg(A.pinmask + D.pin_off + (int64_t)y * D.pin_wpr + (x >> 5)) >> (x & 31)) & 1u;
            float un[3], vn[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                vn[k] = pinned ? pin_v(D, k) : fmaf(D.dt_net, a3[k], sU[3 + k][yy][sx]);
                un[k] = fmaf(D.dt_net, vn[k], sU[k][yy][sx]);
            }
            if (D.sph_on) sphere_contact(D, x, y, h, un[0], un[1], un[2], vn[0], vn[1], vn[2]);
            if (!isfinite(un[0] + un[1] + un[2])) atomicOr(A.status, kStatusNonfinite);
            float* out = A.dst + D.plane_off + (int64_t)y * D.pitch + col_pos(x);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                out[k * D.plane_stride] = un[k];
                out[(3 + k) * D.plane_stride] = vn[k];
            }
        }
    }
}

}  // namespace

int pcell_tile_rows() { return TH; }
int pcell_tile_cols() { return TW; }

cudaError_t launch_pcell(const ClothDesc* desc, const int4* tiles, int n_tiles, const float* w, const float* src,
                         float* dst, float* a_out, const uint32_t* pinmask, int32_t* status, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    PcellArgs a{};
    a.desc = desc;
    a.tiles = tiles;
    a.w = w;
    a.src = src;
    a.dst = dst;
    a.a_out = a_out;
    a.pinmask = pinmask;
    a.status = status;
    if (a_out) pcell_kernel<false><<<n_tiles, NT, 0, s>>>(a);
    else pcell_kernel<true><<<n_tiles, NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace cloth
