// Plain mass-spring step (Sec. 3.1, Eq. 1-5), scalar FP32 variant used when
// any cloth of the batch has spring-axis damping (Eq. 2, mu != 0): it also
// carries the neighbours' velocities.  The paired-FP32 kernel of
// plain_step.cu serves every batch without spring damping.
//
// Mapping: one warp per work unit (cloth b, strip of kStripDamp = 120 output
// columns, output rows [r0, r1)).  Lane l holds the 4 consecutive columns
// c0 - 4 + 4l .. c0 - 1 + 4l as float4 loads of the SoA planes.  The warp
// marches down the rows with a register window of 4 position rows
// (r-1 .. r+2).  At row r every node evaluates its 6 "forward" springs
// (E, 2E, N, 2N, NE, NW); the reaction -F goes to the partner's accumulator
// either in registers (same lane, rows r..r+2) or through one warp shuffle
// (neighbour lane).  After row r's springs, its force accumulator holds all
// 12 springs (the backward ones arrived from rows r-2, r-1 and from the left
// lane), so the node is finished: pressure (Eq. 3), gravity and drag
// (Eq. 4), the semi-implicit Euler update with pins (Eq. 5) and sphere
// contact, then the float4 store.  Each spring is evaluated once, with
// 1 rsqrt and 1 fast division.
//
// Precision: positions are stored as u = x - X (displacement from the rest
// lattice).  A spring's vector is d = l + du with l the exact lattice
// offset (multiples of h) and du = u_j - u_i, and its stretch uses
// |d|^2 - L^2 = du . (2 l + du) (since |l| = L), so (|d| - L) / |d| =
// (|d|^2 - L^2) / (|d| (|d| + L)) carries no cancellation in FP32.
#include "cloth_internal.cuh"

namespace cloth {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int NC>
struct Row {
    float c[NC][4];  // [component][column]
};

template <int NC>
struct Node {
    float c[NC];
};

template <int NC>
__device__ __forceinline__ void zero(Row<NC>& r)
{
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) r.c[c][k] = 0.f;
}

// Load NC planes (starting at plane `plane0`) of one row of 4 columns.
template <int NC>
__device__ __forceinline__ void load_row(Row<NC>& r, const float* base, int64_t stride, int plane0, bool ok)
{
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok) t = __ldg(reinterpret_cast<const float4*>(base + (int64_t)(plane0 + c) * stride));
        const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) r.c[c][k] = tv[col_slot(k)];
    }
}

template <int NC>
__device__ __forceinline__ Node<NC> at(const Row<NC>& r, int k)
{
    Node<NC> n;
#pragma unroll
    for (int c = 0; c < NC; ++c) n.c[c] = r.c[c][k];
    return n;
}

// Column k of the neighbour lane (delta = +1: lane + 1, delta = -1: lane - 1).
template <int NC>
__device__ __forceinline__ Node<NC> from_lane(const Row<NC>& r, int k, int delta)
{
    Node<NC> n;
#pragma unroll
    for (int c = 0; c < NC; ++c)
        n.c[c] = delta > 0 ? __shfl_down_sync(kFull, r.c[c][k], 1) : __shfl_up_sync(kFull, r.c[c][k], 1);
    return n;
}

// Force on node i from the spring (i, j) with lattice offset (lx, ly, 0) =
// X_j - X_i and rest length L: Eq. 1 with x_ij = x_i - x_j gives
// f_i = k (|d| - L) d / |d|, d = x_j - x_i; Eq. 2 adds mu ((v_j - v_i) . d) d / |d|^2.
template <int NC>
__device__ __forceinline__ float3 spring(float lx, float ly, float L, float k, float mu, const Node<NC>& i,
                                         const Node<NC>& j, bool ok)
{
    const float dux = j.c[0] - i.c[0], duy = j.c[1] - i.c[1], duz = j.c[2] - i.c[2];
    const float dx = lx + dux, dy = ly + duy, dz = duz;
    const float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float num = fmaf(dux, dx + lx, fmaf(duy, dy + ly, duz * dz));   // |d|^2 - L^2
    const float rq = rsqrt_ftz(q);
    float s = k * num * rq * rcp_ftz(fmaf(q, rq, L));
    if constexpr (NC == 6) {
        const float dvx = j.c[3] - i.c[3], dvy = j.c[4] - i.c[4], dvz = j.c[5] - i.c[5];
        s = fmaf(mu * fmaf(dvx, dx, fmaf(dvy, dy, dvz * dz)), rq * rq, s);
    }
    s = ok ? s : 0.f;
    return make_float3(s * dx, s * dy, s * dz);
}

__device__ __forceinline__ void add3(float (&a)[3][4], int k, float3 f)
{
    a[0][k] += f.x; a[1][k] += f.y; a[2][k] += f.z;
}
__device__ __forceinline__ void sub3(float (&a)[3][4], int k, float3 f)
{
    a[0][k] -= f.x; a[1][k] -= f.y; a[2][k] -= f.z;
}
__device__ __forceinline__ float3 shfl3_up(float3 f)
{
    return make_float3(__shfl_up_sync(kFull, f.x, 1), __shfl_up_sync(kFull, f.y, 1), __shfl_up_sync(kFull, f.z, 1));
}
__device__ __forceinline__ float3 shfl3_down(float3 f)
{
    return make_float3(__shfl_down_sync(kFull, f.x, 1), __shfl_down_sync(kFull, f.y, 1),
                       __shfl_down_sync(kFull, f.z, 1));
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 fma3(float s, float3 a, float3 b)
{
    return make_float3(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z));
}

template <bool DAMP, bool FORCES>
__global__ void __launch_bounds__(128, 3) plain_step_damp_kernel(StepArgs a)
{
    constexpr int NC = DAMP ? 6 : 3;
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const bool out_lane = lane >= 1 && lane <= 30;

    if (gwarp >= a.n_warps) return;
    for (int u = a.warp_first[gwarp]; u < a.warp_first[gwarp + 1]; ++u) {
        const WorkUnit wu = a.units[u];
        if (a.mode && a.mode[wu.b] != kModePlain) continue;   // stepped by the network
        const ClothDesc& D = a.desc[wu.b];
        const int rows = D.rows, cols = D.cols, pitch = D.pitch;
        const int64_t stride = D.plane_stride;
        const float h = D.h, h2 = 2.f * D.h, hd = 1.41421356237309515f * D.h;
        const float ks = D.k_struct, ksh = D.k_shear, kb = D.k_bend, mu = D.mu;
        const int c4 = wu.c0 - 4 + 4 * lane;
        const bool lane_in = c4 >= 0 && c4 < pitch;
        // bit j of cm: column c4 - 1 + j exists (j = 0..6)
        unsigned cm = 0;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const int col = c4 - 1 + j;
            cm |= (col >= 0 && col < cols) ? (1u << j) : 0u;
        }
        const int64_t lane_off = D.plane_off + (lane_in ? c4 : 0);
        const float* src = a.src + lane_off;
        auto rok = [&](int q) { return (unsigned)q < (unsigned)rows; };
        auto rowp = [&](int q) { return src + (int64_t)(rok(q) ? q : 0) * pitch; };

        const int rb = wu.r0 - 2;
        Row<NC> P1, P2, P3;  // rows r, r+1, r+2 (u, and v when DAMP)
        load_row(P1, rowp(rb), stride, 0, lane_in && rok(rb));
        load_row(P2, rowp(rb + 1), stride, 0, lane_in && rok(rb + 1));
        load_row(P3, rowp(rb + 2), stride, 0, lane_in && rok(rb + 2));
        // own velocity of row r (needed for the update; in P1 when DAMP)
        Row<3> VC, VN;
        if constexpr (!DAMP) load_row(VC, rowp(rb), stride, 3, lane_in && rok(rb));
        float A1[3][4], A2[3][4], A3[3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) A1[c][k] = A2[c][k] = A3[c][k] = 0.f;

        for (int r = rb; r < wu.r1; ++r) {
            // prefetch row r+3 and (no damping) the velocity of row r+1
            Row<NC> P4;
            load_row(P4, rowp(r + 3), stride, 0, lane_in && rok(r + 3));
            if constexpr (!DAMP) load_row(VN, rowp(r + 1), stride, 3, lane_in && rok(r + 1));

            const bool ok_r = rok(r), ok_r1 = rok(r + 1), ok_r2 = rok(r + 2);
            // neighbour-lane columns: lane+1's columns 0, 1 of row r, column 0
            // of row r+1; lane-1's column 3 of row r+1
            const Node<NC> Ra1 = from_lane(P1, 0, +1), Rb1 = from_lane(P1, 1, +1);
            const Node<NC> Ra2 = from_lane(P2, 0, +1), L2 = from_lane(P2, 3, -1);
            float3 sendA_r = make_float3(0.f, 0.f, 0.f), sendB_r = sendA_r, sendA_r1 = sendA_r, sendD_r1 = sendA_r;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const Node<NC> ni = at(P1, k);
                const bool own = ok_r && ((cm >> (k + 1)) & 1u);
                const bool cE = (cm >> (k + 2)) & 1u, c2E = (cm >> (k + 3)) & 1u, cW = (cm >> k) & 1u;
                const Node<NC> pE = k < 3 ? at(P1, k < 3 ? k + 1 : 0) : Ra1;
                const Node<NC> p2E = k < 2 ? at(P1, k < 2 ? k + 2 : 0) : (k == 2 ? Ra1 : Rb1);
                const Node<NC> pN = at(P2, k), p2N = at(P3, k);
                const Node<NC> pNE = k < 3 ? at(P2, k < 3 ? k + 1 : 0) : Ra2;
                const Node<NC> pNW = k > 0 ? at(P2, k > 0 ? k - 1 : 0) : L2;
                const float3 fE = spring(h, 0.f, h, ks, mu, ni, pE, own && cE);
                const float3 f2E = spring(h2, 0.f, h2, kb, mu, ni, p2E, own && c2E);
                const float3 fN = spring(0.f, h, h, ks, mu, ni, pN, own && ok_r1);
                const float3 f2N = spring(0.f, h2, h2, kb, mu, ni, p2N, own && ok_r2);
                const float3 fNE = spring(h, h, hd, ksh, mu, ni, pNE, own && ok_r1 && cE);
                const float3 fNW = spring(-h, h, hd, ksh, mu, ni, pNW, own && ok_r1 && cW);
                add3(A1, k, make_float3(fE.x + f2E.x + fN.x + f2N.x + fNE.x + fNW.x,
                                        fE.y + f2E.y + fN.y + f2N.y + fNE.y + fNW.y,
                                        fE.z + f2E.z + fN.z + f2N.z + fNE.z + fNW.z));
                sub3(A2, k, fN);
                sub3(A3, k, f2N);
                if (k < 3) sub3(A1, k < 3 ? k + 1 : 0, fE);
                else sendA_r = make_float3(sendA_r.x + fE.x, sendA_r.y + fE.y, sendA_r.z + fE.z);
                if (k < 2) sub3(A1, k < 2 ? k + 2 : 0, f2E);
                else if (k == 2) sendA_r = make_float3(sendA_r.x + f2E.x, sendA_r.y + f2E.y, sendA_r.z + f2E.z);
                else sendB_r = f2E;
                if (k < 3) sub3(A2, k < 3 ? k + 1 : 0, fNE);
                else sendA_r1 = fNE;
                if (k > 0) sub3(A2, k > 0 ? k - 1 : 0, fNW);
                else sendD_r1 = fNW;
            }
            sub3(A1, 0, shfl3_up(sendA_r));
            sub3(A1, 1, shfl3_up(sendB_r));
            sub3(A2, 0, shfl3_up(sendA_r1));
            sub3(A2, 3, shfl3_down(sendD_r1));

            // pressure (Eq. 3) of row r+1, whose 4 cardinal neighbours are in
            // rows r .. r+2 of the window, goes into its accumulator
            if (D.p_quarter != 0.f && ok_r1) {
                const float pq = D.p_quarter;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const Node<NC> ni = at(P2, k);
                    const Node<NC> nE = k < 3 ? at(P2, k < 3 ? k + 1 : 0) : Ra2;
                    const Node<NC> nW = k > 0 ? at(P2, k > 0 ? k - 1 : 0) : L2;
                    const Node<NC> nN = at(P3, k), nS = at(P1, k);
                    const bool bE = (cm >> (k + 2)) & 1u, bW = (cm >> k) & 1u;
                    const float3 dE = make_float3(h + nE.c[0] - ni.c[0], nE.c[1] - ni.c[1], nE.c[2] - ni.c[2]);
                    const float3 dW = make_float3(-h + nW.c[0] - ni.c[0], nW.c[1] - ni.c[1], nW.c[2] - ni.c[2]);
                    const float3 dN = make_float3(nN.c[0] - ni.c[0], h + nN.c[1] - ni.c[1], nN.c[2] - ni.c[2]);
                    const float3 dS = make_float3(nS.c[0] - ni.c[0], -h + nS.c[1] - ni.c[1], nS.c[2] - ni.c[2]);
                    float3 T = make_float3(0.f, 0.f, 0.f);
                    T = fma3((bE && ok_r2) ? 1.f : 0.f, cross3(dE, dN), T);
                    T = fma3((ok_r2 && bW) ? 1.f : 0.f, cross3(dN, dW), T);
                    T = fma3((bW && ok_r) ? 1.f : 0.f, cross3(dW, dS), T);
                    T = fma3((ok_r && bE) ? 1.f : 0.f, cross3(dS, dE), T);
                    add3(A2, k, make_float3(pq * T.x, pq * T.y, pq * T.z));
                }
            }

            // row r is complete: gravity and drag, update, store
            if (r >= wu.r0 && ok_r && out_lane && ((cm >> 1) & 1u)) {
                const ClothDesc& Dd = D;
                float vx[4], vy[4], vz[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if constexpr (DAMP) { vx[k] = P1.c[3][k]; vy[k] = P1.c[4][k]; vz[k] = P1.c[5][k]; }
                    else { vx[k] = VC.c[0][k]; vy[k] = VC.c[1][k]; vz[k] = VC.c[2][k]; }
                }
                float fx[4], fy[4], fz[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    fx[k] = A1[0][k] + fmaf(-Dd.drag, vx[k], Dd.m * Dd.gx);
                    fy[k] = A1[1][k] + fmaf(-Dd.drag, vy[k], Dd.m * Dd.gy);
                    fz[k] = A1[2][k] + fmaf(-Dd.drag, vz[k], Dd.m * Dd.gz);
                }
                if constexpr (FORCES) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int col = c4 + k;
                        if (col < cols) {
                            float* o = a.force_out + (Dd.abi_off + (int64_t)r * cols + col) * 3;
                            o[0] = fx[k]; o[1] = fy[k]; o[2] = fz[k];
                        }
                    }
                } else {
                    const uint32_t pw = __ldg(a.pinmask + Dd.pin_off + (int64_t)r * Dd.pin_wpr + (c4 >> 5));
                    const unsigned pbits = (pw >> (c4 & 31)) & 0xfu;
                    const float dt = Dd.dt, dtm = Dd.dt * Dd.inv_m;
                    float un[3][4], vn[3][4];
                    bool finite = true;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool pinned = (pbits >> k) & 1u;
                        float nvx = fmaf(dtm, fx[k], vx[k]), nvy = fmaf(dtm, fy[k], vy[k]), nvz = fmaf(dtm, fz[k], vz[k]);
                        if (pinned) {   // C: the velocity of the object the node moves with
                            nvx = Dd.pin_vx;
                            nvy = Dd.pin_vy;
                            nvz = Dd.pin_vz;
                        }
                        float nux = fmaf(dt, nvx, P1.c[0][k]), nuy = fmaf(dt, nvy, P1.c[1][k]), nuz = fmaf(dt, nvz, P1.c[2][k]);
                        if (Dd.sph_on) sphere_contact(Dd, c4 + k, r, h, nux, nuy, nuz, nvx, nvy, nvz);
                        un[0][k] = nux; un[1][k] = nuy; un[2][k] = nuz;
                        vn[0][k] = nvx; vn[1][k] = nvy; vn[2][k] = nvz;
                        if ((cm >> (k + 1)) & 1u)
                            finite = finite && isfinite(nux + nuy + nuz + nvx + nvy + nvz);
                    }
                    if (!finite) atomicOr(a.status, 1);
                    float* dst = a.dst + lane_off + (int64_t)r * pitch;
                    if (c4 + 3 < cols) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float ou[4], ov[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                ou[col_slot(k)] = un[c][k];
                                ov[col_slot(k)] = vn[c][k];
                            }
                            *reinterpret_cast<float4*>(dst + c * stride) = make_float4(ou[0], ou[1], ou[2], ou[3]);
                            *reinterpret_cast<float4*>(dst + (c + 3) * stride) = make_float4(ov[0], ov[1], ov[2], ov[3]);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (c4 + k < cols) {
                                const int m = col_slot(k);
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    dst[c * stride + m] = un[c][k];
                                    dst[(c + 3) * stride + m] = vn[c][k];
                                }
                            }
                    }
                }
            }

            // slide the window down one row
            P1 = P2; P2 = P3; P3 = P4;
            if constexpr (!DAMP) VC = VN;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int k = 0; k < 4; ++k) { A1[c][k] = A2[c][k]; A2[c][k] = A3[c][k]; A3[c][k] = 0.f; }
        }
    }
}

}  // namespace

int plain_step_blocks_per_sm_nodamp(int block);   // plain_step.cu

int plain_step_blocks_per_sm(bool damp, int block)
{
    if (!damp) return plain_step_blocks_per_sm_nodamp(block);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, plain_step_damp_kernel<true, false>, block, 0) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_plain_step_damp(const StepArgs& a, bool forces_only, int grid, int block, cudaStream_t s)
{
    if (forces_only) plain_step_damp_kernel<true, true><<<grid, block, 0, s>>>(a);
    else plain_step_damp_kernel<true, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace cloth
