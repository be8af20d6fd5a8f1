// Plain mass-spring step (Sec. 3.1, Eq. 1-5) for a batch of cloths of
// uneven sizes in one launch, in paired FP32 (f32x2) arithmetic.  Serves
// every batch without spring-axis damping (mu = 0; plain_step_damp.cu
// handles mu != 0).
//
// Mapping: one warp per work unit (cloth b, strip of kStrip = 120 output
// columns, output rows [r0, r1)).  Lane l holds the 4 consecutive columns
// c = c4 .. c4 + 3 (c4 = c0 - 4 + 4 l) as the column pairs A = (c0, c2) and
// B = (c1, c3); lanes 1..30 own the output columns, lanes 0 and 31 are halo
// lanes.  The warp marches down the rows with a register window of the
// position rows r .. r+2 (r+3 in flight).  At row r each node evaluates its
// 6 "forward" springs (E, 2E, N, 2N, NE, NW) once, as 12 spring pairs of
// one type on (c0, c2) or (c1, c3); the reaction -F lands in the partner's
// accumulator, in registers (same lane, rows r .. r+2) or through one warp
// shuffle (neighbour lane).  After row r its accumulator holds all 12
// springs, and the node is finished: gravity and drag (Eq. 4), the
// semi-implicit Euler update (Eq. 5), sphere contact, float4 stores.  The
// pinned nodes (the constraint C of Eq. 5) are set afterwards by a small
// kernel over the pin list (pin_fix_kernel): a per-row test of the pin mask
// inside this kernel cost about 7 % of the step, for a few nodes per cloth.  Pressure (Eq. 3) of row r+1 is added while rows r .. r+2 are in
// the window.
//
// Precision: positions are stored as u = x - X (displacement from the rest
// lattice).  A spring's vector is d = l + du with l the lattice offset and
// du = u_j - u_i, and its stretch uses |d|^2 - L^2 = du . (2 l + du) (since
// |l| = L), so (|d| - L) / |d| = (|d|^2 - L^2) / (|d| (|d| + L)) carries no
// cancellation in FP32.
#include <type_traits>

#include "cloth_internal.cuh"

// Resident blocks of 128 threads per SM the register budget is sized for.
#ifndef CLOTH_PLAIN_MINB
#define CLOTH_PLAIN_MINB 3
#endif

namespace cloth {
namespace {

constexpr unsigned kFull = 0xffffffffu;
using f2 = float2;

__device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start before the kernel ahead of it in the stream has
// finished; it waits for that kernel (and its memory) before it touches the
// state, and lets the next one launch at once.  Without the launch
// attribute both are no-ops.
__device__ __forceinline__ void pdl_wait_then_release()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, F2(-1.f), a); }   // a - b, one rounding

// One row of a lane: the column pairs A = (c0, c2) and B = (c1, c3) of the
// three components.
struct Row2 {
    f2 A[3], B[3];
};

__device__ __forceinline__ void zero(Row2& r)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) r.A[c] = r.B[c] = F2(0.f);
}

// Planes plane0 .. plane0+2 of one row; memory order c0 c2 c1 c3.
__device__ __forceinline__ void load2(Row2& r, const float* base, int64_t stride, int plane0, bool ok)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok) t = __ldg(reinterpret_cast<const float4*>(base + (int64_t)(plane0 + c) * stride));
        r.A[c] = make_float2(t.x, t.y);
        r.B[c] = make_float2(t.z, t.w);
    }
}

// Lattice offset S h along one axis as a pair (S in {-1, 1, 2}).
template <int S>
__device__ __forceinline__ f2 lat(f2 h, f2 h2, f2 nh)
{
    static_assert(S == 1 || S == 2 || S == -1, "lattice offset");
    return S == 1 ? h : (S == 2 ? h2 : nh);
}

// Spring pair of lattice offset (SX, SY) h: returns s with f_i = s d and
// f_j = -s d, d = x_j - x_i (written to d).  Eq. 1 with x_ij = x_i - x_j
// gives s = k (|d| - L) / |d| = k (|d|^2 - L^2) / (|d| (|d| + L)).  The
// stiffness pair k is 0 in a half whose spring does not exist, which gives
// s = 0 there: partner slots outside the grid hold finite values (zero fill
// or the zeroed padding columns), so |d| is finite and non-zero.
template <int SX, int SY>
__device__ __forceinline__ f2 spring2(const f2 (&ui)[3], const f2 (&uj)[3], f2 h, f2 h2, f2 nh, f2 L, f2 L2, f2 k,
                                      f2 (&d)[3])
{
    const f2 dux = sub2(uj[0], ui[0]), duy = sub2(uj[1], ui[1]), duz = sub2(uj[2], ui[2]);
    f2 num;
    if constexpr (SX != 0) {
        const f2 lx = lat<SX>(h, h2, nh);
        d[0] = add2(lx, dux);
        num = mul2(dux, add2(d[0], lx));
    } else {
        d[0] = dux;
        num = mul2(dux, dux);
    }
    if constexpr (SY != 0) {
        const f2 ly = lat<SY>(h, h2, nh);
        d[1] = add2(ly, duy);
        num = fma2(duy, add2(d[1], ly), num);
    } else {
        d[1] = duy;
        num = fma2(duy, duy, num);
    }
    d[2] = duz;
    num = fma2(duz, duz, num);                       // |d|^2 - L^2
    const f2 q = add2(num, L2);                      // |d|^2
    const f2 rq = make_float2(rsqrt_ftz(q.x), rsqrt_ftz(q.y));
    const f2 den = fma2(q, rq, L);                   // |d| + L
    const f2 t = mul2(mul2(k, num), rq);
    return mul2(t, make_float2(rcp_ftz(den.x), rcp_ftz(den.y)));
}

__device__ __forceinline__ void acc2(f2 (&a)[3], f2 s, const f2 (&d)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) a[c] = fma2(s, d[c], a[c]);
}
__device__ __forceinline__ float shup(float v) { return __shfl_up_sync(kFull, v, 1); }
__device__ __forceinline__ float shdn(float v) { return __shfl_down_sync(kFull, v, 1); }

// Per-warp constants of the current unit for the update (Eq. 4-5): read
// from shared memory where they are used, instead of being held in
// registers through the spring arithmetic or re-read from the descriptor
// in global memory after every row's stores.
struct UnitConst {
    float dt, dtm, keep, dtg[3];   // dt, dt/m, 1 - dt d/m, dt g
    int32_t sph_on;
};

// Stiffness pairs of the 12 springs a lane evaluates per row, indexed
// [spring][thread]: E, 2E, N, 2N, NE, NW of pair A, then of pair B.
enum { kE, kT, kN, k2N, kNE, kNW };
constexpr int kSprings = 12;

template <bool FORCES>
__global__ void __launch_bounds__(128, CLOTH_PLAIN_MINB) plain_step_kernel(StepArgs a)
{
    // Each entry is k where the spring exists and 0 elsewhere: the column
    // part is fixed per work unit, the row part changes only in the first
    // and last rows of a cloth.  Kept in shared memory (12 KB per block)
    // rather than registers or per-spring selects.
    __shared__ float2 s_kp[kSprings][128];
    // Pressure coefficients of the lane's pairs A and B (Eq. 3, scaled by
    // p/4): E and W masks, the own-node weight -(mE + mW), and the lattice
    // part of d'_E - d'_W along x.
    __shared__ float2 s_pc[8][128];
    __shared__ UnitConst s_uc[4];
    const int lane = threadIdx.x & 31;
    float2* kp = &s_kp[0][threadIdx.x];
    float2* pc = &s_pc[0][threadIdx.x];
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const bool out_lane = lane >= 1 && lane <= 30;

    pdl_wait_then_release();
    if (gwarp >= a.n_warps) return;
    for (int u = a.warp_first[gwarp]; u < a.warp_first[gwarp + 1]; ++u) {
        const WorkUnit wu = a.units[u];
        if (a.mode && a.mode[wu.b] != kModePlain) continue;   // stepped by the network
        const ClothDesc& D = a.desc[wu.b];
        const int rows = D.rows, cols = D.cols, pitch = D.pitch;
        const int64_t stride = D.plane_stride;
        const int c4 = wu.c0 - 4 + 4 * lane;
        const bool lane_in = c4 >= 0 && c4 < pitch;
        // bit j of cm: column c4 - 1 + j exists (j = 0..6)
        unsigned cm = 0;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const int col = c4 - 1 + j;
            cm |= (col >= 0 && col < cols) ? (1u << j) : 0u;
        }
        auto bit = [&](int j) { return ((cm >> j) & 1u) != 0u; };
        const bool oA0 = bit(1);   // column c4 exists
        const float hs = D.h;
        const float pq = D.p_quarter;
        volatile UnitConst* uc = &s_uc[threadIdx.x >> 5];
        if (lane == 0) {
            uc->dt = D.dt;
            uc->dtm = D.dt * D.inv_m;
            uc->keep = 1.f - D.dt * D.inv_m * D.drag;
            uc->dtg[0] = D.dt * D.gx;
            uc->dtg[1] = D.dt * D.gy;
            uc->dtg[2] = D.dt * D.gz;
            uc->sph_on = D.sph_on;
        }
        __syncwarp();
        {
            // pressure masks: the E neighbour of each half exists (mE) / the
            // W neighbour exists (mW, stored negated)
            auto put = [&](int j, float e0, float e1, float w0, float w1) {
                pc[(4 * j + 0) * 128] = make_float2(pq * e0, pq * e1);
                pc[(4 * j + 1) * 128] = make_float2(-pq * w0, -pq * w1);
                pc[(4 * j + 2) * 128] = make_float2(pq * (w0 - e0), pq * (w1 - e1));
                pc[(4 * j + 3) * 128] = make_float2(pq * (e0 + w0) * hs, pq * (e1 + w1) * hs);
            };
            auto m = [&](int j) { return bit(j) ? 1.f : 0.f; };
            put(0, m(2), m(4), m(0), m(2));   // A = (c0, c2): E c1, c3; W c-1, c1
            put(1, m(3), m(5), m(1), m(3));   // B = (c1, c3): E c2, c4; W c0, c2
        }
        const f2 h = F2(hs), h2 = F2(2.f * hs), nh = F2(-hs);
        const f2 Ls = F2(hs), Ls2 = F2(hs * hs), Lb = F2(2.f * hs), Lb2 = F2(4.f * hs * hs);
        const f2 Ld = F2(1.41421356237309515f * hs), Ld2 = F2(2.f * hs * hs);
        // stiffness pairs with the column part of each spring's existence
        // (own node and partner in the grid's columns); `rows_on` adds the
        // row part: springs reaching row r+1 (N) or r+2 (2N) exist only
        // while that row does, and a row above the grid owns none
        auto set_kp = [&](bool row_r, bool row_r1, bool row_r2) {
            auto pr = [&](float k, bool on, int o0, int p0, int o1, int p1) {
                return make_float2(on && bit(o0) && bit(p0) ? k : 0.f, on && bit(o1) && bit(p1) ? k : 0.f);
            };
            const float ks = D.k_struct, ksh = D.k_shear, kb = D.k_bend;
            const bool n1 = row_r && row_r1, n2 = row_r && row_r2;
            kp[(0 + kE) * 128] = pr(ks, row_r, 1, 2, 3, 4);   // A: partners c1, c3
            kp[(0 + kT) * 128] = pr(kb, row_r, 1, 3, 3, 5);   //    c2, c4
            kp[(0 + kN) * 128] = pr(ks, n1, 1, 1, 3, 3);
            kp[(0 + k2N) * 128] = pr(kb, n2, 1, 1, 3, 3);
            kp[(0 + kNE) * 128] = pr(ksh, n1, 1, 2, 3, 4);
            kp[(0 + kNW) * 128] = pr(ksh, n1, 1, 0, 3, 2);    //    c-1, c1
            kp[(6 + kE) * 128] = pr(ks, row_r, 2, 3, 4, 5);   // B: partners c2, c4
            kp[(6 + kT) * 128] = pr(kb, row_r, 2, 4, 4, 6);   //    c3, c5
            kp[(6 + kN) * 128] = pr(ks, n1, 2, 2, 4, 4);
            kp[(6 + k2N) * 128] = pr(kb, n2, 2, 2, 4, 4);
            kp[(6 + kNE) * 128] = pr(ksh, n1, 2, 3, 4, 5);
            kp[(6 + kNW) * 128] = pr(ksh, n1, 2, 1, 4, 3);    //    c0, c2
        };
        auto K = [&](int j) { return kp[j * 128]; };
        const int64_t lane_off = D.plane_off + (lane_in ? c4 : 0);
        const float* src = a.src + lane_off;
        auto rok = [&](int q) { return (unsigned)q < (unsigned)rows; };
        auto rowp = [&](int q) { return src + (int64_t)(rok(q) ? q : 0) * pitch; };

        const int rb = wu.r0 - 2;
        set_kp(rok(rb), rok(rb + 1), rok(rb + 2));
        Row2 P0, P1, P2, F0, F1, Fq;   // rows r, r+1, r+2; forces of r, r+1, r+2
        load2(P0, rowp(rb), stride, 0, lane_in && rok(rb));
        load2(P1, rowp(rb + 1), stride, 0, lane_in && rok(rb + 1));
        load2(P2, rowp(rb + 2), stride, 0, lane_in && rok(rb + 2));
        zero(F0); zero(F1); zero(Fq);

        // One row of the march.  kMode 2: an output row.  The two warm-up
        // rows above the unit (kMode 0: r0 - 2, kMode 1: r0 - 1) only feed the
        // accumulators of rows r0 and r0 + 1, so they evaluate only the springs
        // that reach those rows (row r0 - 2: 2N; row r0 - 1: N, 2N, NE, NW) and
        // the pressure of row r0; the output rows see the same contributions in
        // the same order either way.
        auto row = [&](auto mode_tag, const int r) {
            constexpr int kMode = decltype(mode_tag)::value;
            // positions of row r+3 are needed next row; the velocity of row r
            // only at the end of this one: both loads have a row of work to land
            Row2 PN, V0;
            load2(PN, rowp(r + 3), stride, 0, lane_in && rok(r + 3));
            if constexpr (kMode == 2) load2(V0, rowp(r), stride, 3, lane_in && rok(r) && out_lane);

            const bool ok_r = rok(r), ok_r1 = rok(r + 1), ok_r2 = rok(r + 2);
            // the row part of the stiffness pairs changes only at a cloth's
            // first two rows (the top halo ends) and last two rows
            if (r > rb && (r <= 0 || !ok_r2)) set_kp(ok_r, ok_r1, ok_r2);
            // assembled partner pairs (per component):
            //   X0 = (c2, c4) of row r, Y0 = (c3, c5) of row r,
            //   X1 = (c2, c4) of row r+1, Z1 = (c-1, c1) of row r+1
            f2 X0[3], Y0[3], X1[3], Z1[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if constexpr (kMode == 2) {
                    X0[c] = make_float2(P0.A[c].y, shdn(P0.A[c].x));
                    Y0[c] = make_float2(P0.B[c].y, shdn(P0.B[c].x));
                }
                if constexpr (kMode >= 1) {
                    X1[c] = make_float2(P1.A[c].y, shdn(P1.A[c].x));
                    Z1[c] = make_float2(shup(P1.B[c].y), P1.B[c].x);
                }
            }
            f2 d[3], s;
            float sR0r[3] = {0.f, 0.f, 0.f}, sR1r[3] = {0.f, 0.f, 0.f};
            float sR0r1[3] = {0.f, 0.f, 0.f}, sL3r1[3] = {0.f, 0.f, 0.f};

            // ---- springs of the A pair (c0, c2)
            if constexpr (kMode == 2) {
                s = spring2<1, 0>(P0.A, P0.B, h, h2, nh, Ls, Ls2, K(0 + kE), d);      // E -> (c1, c3)
                acc2(F0.A, s, d);
                acc2(F0.B, mul2(s, F2(-1.f)), d);
                s = spring2<2, 0>(P0.A, X0, h, h2, nh, Lb, Lb2, K(0 + kT), d);        // 2E -> (c2, c4)
                acc2(F0.A, s, d);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const f2 f = mul2(s, d[c]);
                    F0.A[c].y -= f.x;
                    sR0r[c] += f.y;
                }
            }
            if constexpr (kMode >= 1) {
                s = spring2<0, 1>(P0.A, P1.A, h, h2, nh, Ls, Ls2, K(0 + kN), d);        // N
                acc2(F0.A, s, d);
                acc2(F1.A, mul2(s, F2(-1.f)), d);
            }
            s = spring2<0, 2>(P0.A, P2.A, h, h2, nh, Lb, Lb2, K(0 + k2N), d);          // 2N
            acc2(F0.A, s, d);
            acc2(Fq.A, mul2(s, F2(-1.f)), d);
            if constexpr (kMode >= 1) {
                s = spring2<1, 1>(P0.A, P1.B, h, h2, nh, Ld, Ld2, K(0 + kNE), d);       // NE -> (c1, c3)
                acc2(F0.A, s, d);
                acc2(F1.B, mul2(s, F2(-1.f)), d);
                s = spring2<-1, 1>(P0.A, Z1, h, h2, nh, Ld, Ld2, K(0 + kNW), d);        // NW -> (c-1, c1)
                acc2(F0.A, s, d);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const f2 f = mul2(s, d[c]);
                    sL3r1[c] += f.x;
                    F1.B[c].x -= f.y;
                }
            }
            // ---- springs of the B pair (c1, c3)
            if constexpr (kMode == 2) {
                s = spring2<1, 0>(P0.B, X0, h, h2, nh, Ls, Ls2, K(6 + kE), d);        // E -> (c2, c4)
                acc2(F0.B, s, d);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const f2 f = mul2(s, d[c]);
                    F0.A[c].y -= f.x;
                    sR0r[c] += f.y;
                }
                s = spring2<2, 0>(P0.B, Y0, h, h2, nh, Lb, Lb2, K(6 + kT), d);        // 2E -> (c3, c5)
                acc2(F0.B, s, d);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const f2 f = mul2(s, d[c]);
                    F0.B[c].y -= f.x;
                    sR1r[c] += f.y;
                }
            }
            if constexpr (kMode >= 1) {
                s = spring2<0, 1>(P0.B, P1.B, h, h2, nh, Ls, Ls2, K(6 + kN), d);        // N
                acc2(F0.B, s, d);
                acc2(F1.B, mul2(s, F2(-1.f)), d);
            }
            s = spring2<0, 2>(P0.B, P2.B, h, h2, nh, Lb, Lb2, K(6 + k2N), d);          // 2N
            acc2(F0.B, s, d);
            acc2(Fq.B, mul2(s, F2(-1.f)), d);
            if constexpr (kMode >= 1) {
                s = spring2<1, 1>(P0.B, X1, h, h2, nh, Ld, Ld2, K(6 + kNE), d);         // NE -> (c2, c4)
                acc2(F0.B, s, d);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const f2 f = mul2(s, d[c]);
                    F1.A[c].y -= f.x;
                    sR0r1[c] += f.y;
                }
                s = spring2<-1, 1>(P0.B, P1.A, h, h2, nh, Ld, Ld2, K(6 + kNW), d);      // NW -> (c0, c2)
                acc2(F0.B, s, d);
                acc2(F1.A, mul2(s, F2(-1.f)), d);
            }

            // ---- reactions that cross to the neighbour lanes
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if constexpr (kMode == 2) {
                    F0.A[c].x -= shup(sR0r[c]);
                    F0.B[c].x -= shup(sR1r[c]);
                }
                if constexpr (kMode >= 1) {
                    F1.A[c].x -= shup(sR0r1[c]);
                    F1.B[c].y -= shdn(sL3r1[c]);
                }
            }

            // ---- pressure (Eq. 3) of row r+1, whose 4 cardinal neighbours lie
            // in rows r .. r+2.  With d'_n = (neighbour n exists)(x_n - x_i),
            // the sum over the ordered pairs of d'_E x d'_N + d'_N x d'_W +
            // d'_W x d'_S + d'_S x d'_E equals (d'_E - d'_W) x (d'_N - d'_S).
            // d'_E - d'_W = mE x_E + mW x_W - (mE + mW) x_i (mW negated): for
            // an interior node x_i drops out and it is x_E - x_W + 2 h x^.
            if (kMode >= 1 && pq != 0.f && ok_r1) {
                const float fN = ok_r2 ? 1.f : 0.f, fS = ok_r ? 1.f : 0.f;
                const f2 bN = F2(fN), bSn = F2(-fS), cN = F2(fS - fN), hy = F2((fN + fS) * hs);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const f2* ui = half == 0 ? P1.A : P1.B;
                    const f2* uE = half == 0 ? P1.B : X1;
                    const f2* uW = half == 0 ? Z1 : P1.A;
                    const f2* uN = half == 0 ? P2.A : P2.B;
                    const f2* uS = half == 0 ? P0.A : P0.B;
                    // e = (p/4)(d'_E - d'_W), n = d'_N - d'_S
                    const f2 qE = pc[(4 * half + 0) * 128], qW = pc[(4 * half + 1) * 128];
                    const f2 qC = pc[(4 * half + 2) * 128], qh = pc[(4 * half + 3) * 128];
                    const f2 ex = fma2(qE, uE[0], fma2(qW, uW[0], fma2(qC, ui[0], qh)));
                    const f2 ey = fma2(qE, uE[1], fma2(qW, uW[1], mul2(qC, ui[1])));
                    const f2 ez = fma2(qE, uE[2], fma2(qW, uW[2], mul2(qC, ui[2])));
                    const f2 nx = fma2(bN, uN[0], fma2(bSn, uS[0], mul2(cN, ui[0])));
                    const f2 ny = fma2(bN, uN[1], fma2(bSn, uS[1], fma2(cN, ui[1], hy)));
                    const f2 nz = fma2(bN, uN[2], fma2(bSn, uS[2], mul2(cN, ui[2])));
                    auto neg = [](f2 v) { return make_float2(-v.x, -v.y); };
                    f2* Fh = half == 0 ? F1.A : F1.B;
                    Fh[0] = fma2(ey, nz, fma2(neg(ez), ny, Fh[0]));
                    Fh[1] = fma2(ez, nx, fma2(neg(ex), nz, Fh[1]));
                    Fh[2] = fma2(ex, ny, fma2(neg(ey), nx, Fh[2]));
                }
            }

            // ---- row r is complete: gravity and drag (Eq. 4), update (Eq. 5)
            if (kMode == 2 && ok_r && out_lane && oA0) {
                if constexpr (FORCES) {
                    const f2 ndrag = F2(-D.drag);
                    const f2 mg[3] = {F2(D.m * D.gx), F2(D.m * D.gy), F2(D.m * D.gz)};
                    Row2 f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        f.A[c] = add2(F0.A[c], fma2(ndrag, V0.A[c], mg[c]));
                        f.B[c] = add2(F0.B[c], fma2(ndrag, V0.B[c], mg[c]));
                    }
                    float* o = a.force_out + (D.abi_off + (int64_t)r * cols + c4) * 3;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        o[0 * 3 + c] = f.A[c].x;
                        if (c4 + 1 < cols) o[1 * 3 + c] = f.B[c].x;
                        if (c4 + 2 < cols) o[2 * 3 + c] = f.A[c].y;
                        if (c4 + 3 < cols) o[3 * 3 + c] = f.B[c].y;
                    }
                } else {
                    // v' = v + dt/m (f_int + f_p - d v + m g) = dt/m (f_int + f_p)
                    //      + ((1 - d dt/m) v + dt g): Eq. 4-5 with the
                    // constant terms folded
                    const f2 dt = F2(uc->dt), dtm = F2(uc->dtm);
                    const f2 keep = F2(uc->keep);
                    const f2 dtg[3] = {F2(uc->dtg[0]), F2(uc->dtg[1]), F2(uc->dtg[2])};
                    Row2 un, vn;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        vn.A[c] = fma2(dtm, F0.A[c], fma2(keep, V0.A[c], dtg[c]));
                        vn.B[c] = fma2(dtm, F0.B[c], fma2(keep, V0.B[c], dtg[c]));
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        un.A[c] = fma2(dt, vn.A[c], P0.A[c]);
                        un.B[c] = fma2(dt, vn.B[c], P0.B[c]);
                    }
                    if (uc->sph_on) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            // column c4 + k sits in pair A (k even) or B (k odd), half k / 2
                            f2* U = (k & 1) ? un.B : un.A;
                            f2* Vv = (k & 1) ? vn.B : vn.A;
                            float& ux = (k >> 1) ? U[0].y : U[0].x;
                            float& uy = (k >> 1) ? U[1].y : U[1].x;
                            float& uz = (k >> 1) ? U[2].y : U[2].x;
                            float& vx = (k >> 1) ? Vv[0].y : Vv[0].x;
                            float& vy = (k >> 1) ? Vv[1].y : Vv[1].x;
                            float& vz = (k >> 1) ? Vv[2].y : Vv[2].x;
                            sphere_contact(D, c4 + k, r, hs, ux, uy, uz, vx, vy, vz);
                        }
                    }
                    // non-finite check over the 4 nodes' positions (a NaN or
                    // infinite velocity reaches u' = u + dt v' in this step;
                    // columns beyond the grid hold finite values)
                    f2 chk = add2(add2(un.A[0], un.A[1]), add2(un.A[2], un.B[0]));
                    chk = add2(chk, add2(un.B[1], un.B[2]));
                    if (!isfinite(chk.x + chk.y)) atomicOr(a.status, 1);
                    float* dst = a.dst + lane_off + (int64_t)r * pitch;
                    if (c4 + 3 < cols) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            *reinterpret_cast<float4*>(dst + c * stride) =
                                make_float4(un.A[c].x, un.A[c].y, un.B[c].x, un.B[c].y);
                            *reinterpret_cast<float4*>(dst + (c + 3) * stride) =
                                make_float4(vn.A[c].x, vn.A[c].y, vn.B[c].x, vn.B[c].y);
                        }
                    } else {
                        // ragged strip end: memory slots c0 -> 0, c2 -> 1, c1 -> 2, c3 -> 3
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            dst[c * stride + 0] = un.A[c].x;
                            dst[(c + 3) * stride + 0] = vn.A[c].x;
                            if (c4 + 1 < cols) { dst[c * stride + 2] = un.B[c].x; dst[(c + 3) * stride + 2] = vn.B[c].x; }
                            if (c4 + 2 < cols) { dst[c * stride + 1] = un.A[c].y; dst[(c + 3) * stride + 1] = vn.A[c].y; }
                        }
                    }
                }
            }

            // slide the window down one row
            P0 = P1; P1 = P2; P2 = PN;
            F0 = F1; F1 = Fq; zero(Fq);
        };
        row(std::integral_constant<int, 0>{}, rb);
        row(std::integral_constant<int, 1>{}, rb + 1);
        for (int r = wu.r0; r < wu.r1; ++r) row(std::integral_constant<int, 2>{}, r);
    }
}

}  // namespace

// C of Eq. 5 for the pinned nodes of the step src -> dst just taken: the
// velocity of the object they move with, the position update with it, and
// sphere contact, exactly as the update of a free node but for the velocity
// (the same single-rounding FMA), overwriting what the step wrote for them.
// One thread per entry (cloth, node) of the pin list; cloths not in plain
// mode (mode set) are left alone.
__global__ void pin_fix_kernel(const ClothDesc* __restrict__ desc, const int2* __restrict__ pins, int n,
                               const float* __restrict__ src, float* __restrict__ dst, const int32_t* __restrict__ mode,
                               int32_t* __restrict__ status)
{
    pdl_wait_then_release();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 p = pins[i];
    if (mode && mode[p.x] != kModePlain) return;
    const ClothDesc& D = desc[p.x];
    const int r = p.y / D.cols, c = p.y % D.cols;
    const int64_t o = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
    float un[3], vn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        vn[k] = pin_v(D, k);
        un[k] = fmaf(D.dt, vn[k], src[o + k * D.plane_stride]);
    }
    if (D.sph_on) sphere_contact(D, c, r, D.h, un[0], un[1], un[2], vn[0], vn[1], vn[2]);
    if (!isfinite(un[0] + un[1] + un[2] + vn[0] + vn[1] + vn[2])) atomicOr(status, kStatusNonfinite);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dst[o + k * D.plane_stride] = un[k];
        dst[o + (3 + k) * D.plane_stride] = vn[k];
    }
}

// The same from the pin mask (one thread per mask word), for a context whose
// pins do not fit its pin list.
__global__ void pin_fix_mask_kernel(const ClothDesc* __restrict__ desc, int B, const uint32_t* __restrict__ mask,
                                    const float* __restrict__ src, float* __restrict__ dst,
                                    const int32_t* __restrict__ mode, int32_t* __restrict__ status)
{
    pdl_wait_then_release();
    const int b = blockIdx.y;
    if (b >= B || (mode && mode[b] != kModePlain)) return;
    const ClothDesc& D = desc[b];
    const int64_t words = (int64_t)D.rows * D.pin_wpr;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t bits = mask[D.pin_off + w];
        const int r = (int)(w / D.pin_wpr), c0 = (int)(w % D.pin_wpr) * 32;
        while (bits) {
            const int c = c0 + __ffs(bits) - 1;
            bits &= bits - 1;
            const int64_t o = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
            float un[3], vn[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                vn[k] = pin_v(D, k);
                un[k] = fmaf(D.dt, vn[k], src[o + k * D.plane_stride]);
            }
            if (D.sph_on) sphere_contact(D, c, r, D.h, un[0], un[1], un[2], vn[0], vn[1], vn[2]);
            if (!isfinite(un[0] + un[1] + un[2] + vn[0] + vn[1] + vn[2])) atomicOr(status, kStatusNonfinite);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dst[o + k * D.plane_stride] = un[k];
                dst[o + (3 + k) * D.plane_stride] = vn[k];
            }
        }
    }
}

int plain_step_blocks_per_sm_nodamp(int block)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, plain_step_kernel<false>, block, 0) != cudaSuccess) return 0;
    return n;
}

// Launch with programmatic stream serialisation: the kernel's launch overlaps
// the tail of the kernel ahead of it (see pdl_wait_then_release).
template <class... P, class... A>
cudaError_t launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, cudaStream_t s, A... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_plain_step(const StepArgs& a, bool forces_only, int grid, int block, cudaStream_t s)
{
    if (forces_only) {
        plain_step_kernel<true><<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaError_t e = launch_pdl(plain_step_kernel<false>, dim3(grid), dim3(block), s, a);
    if (e != cudaSuccess) return e;
    if (a.n_pins > 0) {
        e = launch_pdl(pin_fix_kernel, dim3((a.n_pins + 127) / 128), dim3(128), s, a.desc, a.pin_list, a.n_pins,
                       a.src, a.dst, a.mode, a.status);
    } else if (a.n_pins < 0) {   // the pins did not fit the list: from the mask
        e = launch_pdl(pin_fix_mask_kernel, dim3(64, (unsigned)a.n_cloths), dim3(128), s, a.desc, a.n_cloths,
                       a.pinmask, a.src, a.dst, a.mode, a.status);
    }
    return e;
}

}  // namespace cloth
