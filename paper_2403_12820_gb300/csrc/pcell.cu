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
// Mapping: one block of 256 threads per 32 x 8 output tile; the tile and a
// 2-node halo of the six state planes are staged in shared memory; one
// thread per node.  phi is formed as l_c + (u_j - u_i) from the stored
// displacements u = x - X (l_c the lattice offset), which keeps the
// difference exact to the rounding of u.  Step mode adds the hard-encoded
// pressure (Eq. 3) and runs Eq. 5 with pins and sphere contact.
#include "cloth_internal.cuh"

namespace cloth {
namespace {

constexpr int TW = 32, TH = 8, HALO = 2;
constexpr int SW = TW + 2 * HALO, SH = TH + 2 * HALO;   // staged tile
constexpr int NT = TW * TH;
constexpr int kPcellBlob = 40;

__constant__ int kChDy[12] = {0, 0, 1, -1, 1, 1, -1, -1, 0, 0, 2, -2};
__constant__ int kChDx[12] = {1, -1, 0, 0, 1, -1, 1, -1, 2, -2, 0, 0};

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

template <bool STEP>
__global__ void __launch_bounds__(NT) pcell_kernel(PcellArgs A)
{
    __shared__ float sU[6][SH][SW];
    __shared__ float sW[kPcellBlob];
    const int4 t = A.tiles[blockIdx.x];
    const ClothDesc& D = A.desc[t.x];
    const int H = D.rows, W = D.cols;
    const int y0 = t.y, x0 = t.z;
    const int tid = threadIdx.x;
    if (tid < kPcellBlob) sW[tid] = A.w[tid];
    const float* src = A.src + D.plane_off;
    for (int e = tid; e < 6 * SH * SW; e += NT) {
        const int p = e / (SH * SW), r = (e / SW) % SH, c = e % SW;
        const int y = y0 - HALO + r, x = x0 - HALO + c;
        float val = 0.f;
        if (y >= 0 && y < H && x >= 0 && x < W) val = __ldg(src + p * D.plane_stride + (int64_t)y * D.pitch + col_pos(x));
        sU[p][r][c] = val;
    }
    __syncthreads();

    const int ty = tid / TW, tx = tid % TW;
    const int y = y0 + ty, x = x0 + tx;
    if (y >= H || x >= W) return;
    const int sy = ty + HALO, sx = tx + HALO;
    const float h = D.h, alpha = sW[39];
    float acc[3] = {sW[36], sW[37], sW[38]};
#pragma unroll
    for (int ch = 0; ch < 12; ++ch) {
        const int dy = kChDy[ch], dx = kChDx[ch];
        if (y + dy < 0 || y + dy >= H || x + dx < 0 || x + dx >= W) continue;
        const float wl = sW[ch], wn = sW[12 + ch], wd = sW[24 + ch];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float lat = k == 0 ? (float)dx * h : (k == 1 ? (float)dy * h : 0.f);
            const float phi = lat + (sU[k][sy + dy][sx + dx] - sU[k][sy][sx]);
            const float xi = sU[3 + k][sy + dy][sx + dx] - sU[3 + k][sy][sx];
            const float s = phi * rsqrtf(fmaf(alpha * phi, phi, 1.f));
            acc[k] = fmaf(wl, phi, fmaf(s, fmaf(wd, xi, wn), acc[k]));
        }
    }
    if constexpr (!STEP) {
        float* o = A.a_out + (D.abi_off + (int64_t)y * W + x) * 3;
        o[0] = acc[0]; o[1] = acc[1]; o[2] = acc[2];
        return;
    } else {
        // pressure (Eq. 3): (p/4) (d'_E - d'_W) x (d'_N - d'_S) with absent
        // neighbours' terms dropped
        if (D.p_quarter != 0.f) {
            const bool bE = x + 1 < W, bW = x > 0, bN = y + 1 < H, bS = y > 0;
            float e[3], n[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float ui = sU[k][sy][sx];
                e[k] = (bE ? sU[k][sy][sx + 1] - ui + (k == 0 ? h : 0.f) : 0.f) -
                       (bW ? sU[k][sy][sx - 1] - ui - (k == 0 ? h : 0.f) : 0.f);
                n[k] = (bN ? sU[k][sy + 1][sx] - ui + (k == 1 ? h : 0.f) : 0.f) -
                       (bS ? sU[k][sy - 1][sx] - ui - (k == 1 ? h : 0.f) : 0.f);
            }
            const float sc = D.p_quarter * D.inv_m;
            acc[0] = fmaf(sc, e[1] * n[2] - e[2] * n[1], acc[0]);
            acc[1] = fmaf(sc, e[2] * n[0] - e[0] * n[2], acc[1]);
            acc[2] = fmaf(sc, e[0] * n[1] - e[1] * n[0], acc[2]);
        }
        const bool pinned = (__ldg(A.pinmask + D.pin_off + (int64_t)y * D.pin_wpr + (x >> 5)) >> (x & 31)) & 1u;
        float un[3], vn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            vn[k] = pinned ? 0.f : fmaf(D.dt, acc[k], sU[3 + k][sy][sx]);
            un[k] = fmaf(D.dt, vn[k], sU[k][sy][sx]);
        }
        if (D.sph_on) {
            const float rx = fmaf((float)x, h, -D.sph_cx) + un[0];
            const float ry = fmaf((float)y, h, -D.sph_cy) + un[1];
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
        if (!isfinite(un[0] + un[1] + un[2])) atomicOr(A.status, kStatusNonfinite);
        float* out = A.dst + D.plane_off + (int64_t)y * D.pitch + col_pos(x);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            out[k * D.plane_stride] = un[k];
            out[(3 + k) * D.plane_stride] = vn[k];
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
