// Internal device-side structures of libcloth (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cloth {

// The plain-step kernel maps one warp to a strip of STRIP output columns:
// lane l holds the 4 consecutive columns c0 - 4 + 4 l .. c0 - 1 + 4 l, so
// lanes 1..30 own the output columns c0 .. c0 + 119 and lanes 0 and 31 are
// halo lanes that supply the springs reaching across the strip border.
constexpr int kLaneCols = 4;
constexpr int kStrip = 120;
constexpr int kStripDamp = kStrip;   // the damped kernel (mu != 0) uses the same strips
// Plane pitch (floats per row) is a multiple of this, so every float4 of a
// lane is 16-byte aligned and lies wholly inside or outside [0, pitch).
constexpr int kPitchAlign = 4;
// Device status word bits (include/cloth.h: CLOTH_STATUS_*).
constexpr int kStatusNonfinite = 1, kStatusTimeout = 2;
// Per-cloth step mode of a network rollout (include/cloth.h: cloth_modes).
constexpr int32_t kModeNet = 0, kModePlain = 1;

// Per-cloth descriptor in device memory (built on the host at create).
struct __align__(16) ClothDesc {
    int32_t rows, cols, pitch, pin_wpr;   // pin_wpr: 32-bit pin words per row
    int64_t plane_off;                    // float offset of plane 0 in a state buffer
    int64_t plane_stride;                 // rows * pitch (floats)
    int64_t pin_off;                      // word offset of the pin bitmask
    int64_t abi_off;                      // node offset in the packed ABI layout
    float h, m, inv_m, dt;
    float k_struct, k_shear, k_bend, mu;
    float drag, p_quarter, gx, gy;
    float gz, sph_cx, sph_cy, sph_cz;
    float sph_r, sph_r2;
    int32_t sph_on;
    float sph_mu;                         // contact friction: < 0 stick, else Coulomb mu
    float pin_vx, pin_vy, pin_vz;         // velocity of the pinned nodes (m/s)
    float dt_net;                         // time step of the network step: stride x dt
};

// Component c of the pinned nodes' velocity.
__host__ __device__ __forceinline__ float pin_v(const ClothDesc& D, int c)
{
    return c == 0 ? D.pin_vx : (c == 1 ? D.pin_vy : D.pin_vz);
}

// Sphere contact after the update (intersection elimination, Sec. 3.1): a
// node found inside the sphere moves to the nearest point of its surface.
// Its velocity stops (sph_mu < 0), or, with n the outward normal, loses the
// approaching normal speed j = max(-v.n, 0), keeps a separating one, and
// loses min(|v_t|, sph_mu j) of its tangential speed (Coulomb friction).
// (col, row): the node's lattice position (rest position (col h, row h, 0));
// u = x - X.
__device__ __forceinline__ void sphere_contact(const ClothDesc& D, int col, int row, float h, float& ux, float& uy,
                                               float& uz, float& vx, float& vy, float& vz)
{
    const float rx = fmaf((float)col, h, -D.sph_cx) + ux;
    const float ry = fmaf((float)row, h, -D.sph_cy) + uy;
    const float rz = uz - D.sph_cz;
    const float dd = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    if (!(dd < D.sph_r2 && dd > 0.f)) return;
    const float inv = rsqrtf(dd);
    const float sc = D.sph_r * inv;
    ux = fmaf(sc, rx, ux - rx);
    uy = fmaf(sc, ry, uy - ry);
    uz = fmaf(sc, rz, uz - rz);
    if (D.sph_mu < 0.f) {
        vx = vy = vz = 0.f;
        return;
    }
    const float nx = rx * inv, ny = ry * inv, nz = rz * inv;
    const float vn = fmaf(vx, nx, fmaf(vy, ny, vz * nz));
    const float tx = fmaf(-vn, nx, vx), ty = fmaf(-vn, ny, vy), tz = fmaf(-vn, nz, vz);
    const float tl = sqrtf(fmaf(tx, tx, fmaf(ty, ty, tz * tz)));
    const float j = fmaxf(-vn, 0.f);
    const float keep = tl > D.sph_mu * j ? 1.f - D.sph_mu * j / tl : 0.f;
    const float vo = fmaxf(vn, 0.f);
    vx = fmaf(vo, nx, keep * tx);
    vy = fmaf(vo, ny, keep * ty);
    vz = fmaf(vo, nz, keep * tz);
}

// One warp's work: cloth `b`, strip starting at output column c0, output
// rows [r0, r1).
struct __align__(16) WorkUnit {
    int32_t b, c0, r0, r1;
};

// State buffer layout: for each cloth, 6 planes (u_x, u_y, u_z, v_x, v_y,
// v_z) of rows x pitch floats at plane_off + k * plane_stride, where
// u = x - X is the displacement from the rest lattice.  Inside every
// aligned group of 4 columns the floats are stored in the order
// c0, c2, c1, c3, so that one float4 load hands a lane its column pairs
// (c0, c2) and (c1, c3) as two float2 registers for paired FP32 arithmetic.
__host__ __device__ constexpr int col_slot(int j) { return j == 1 ? 2 : (j == 2 ? 1 : j); }
__host__ __device__ constexpr int col_pos(int c) { return (c & ~3) + col_slot(c & 3); }

// Hardware reciprocal square root and reciprocal with subnormals flushed:
// squared spring lengths and |d| + L are never subnormal for a cloth, and the
// flush drops the subnormal range fix-up around each approximation.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct StepArgs {
    const ClothDesc* desc;
    const WorkUnit* units;      // grouped by warp: warp w runs units [warp_first[w], warp_first[w + 1])
    const int32_t* warp_first;
    int32_t n_warps;
    const float* src;
    float* dst;
    const uint32_t* pinmask;
    float* force_out;     // forces-only mode: packed ABI layout
    int32_t* status;
    const int32_t* mode;  // if set, only cloths in plain mode are stepped
    // pinned nodes, set after the step by the undamped kernel's launcher:
    // (cloth, node) pairs, n_pins of them (0: none; -1: too many for the
    // list, set from the pin mask of the n_cloths cloths instead)
    const int2* pin_list;
    int32_t n_pins, n_cloths;
};

// Launchers (plain_step.cu, state.cu).
cudaError_t launch_plain_step(const StepArgs& a, bool forces_only, int grid, int block, cudaStream_t s);
cudaError_t launch_plain_step_damp(const StepArgs& a, bool forces_only, int grid, int block, cudaStream_t s);
// The literal cell (pcell.cu): tiles of pcell_tile_rows() x pcell_tile_cols()
// output nodes; a_out set -> the cell's acceleration into a_out (packed ABI
// order), else one network step src -> dst.
int pcell_tile_rows();
int pcell_tile_cols();
cudaError_t launch_pcell(const ClothDesc* desc, const int4* tiles, int n_tiles, const float* w, const float* src,
                         float* dst, float* a_out, const uint32_t* pinmask, int32_t* status, cudaStream_t s);
// Blocks of `block` threads of the plain-step kernel resident per SM.
int plain_step_blocks_per_sm(bool damp, int block);
cudaError_t launch_set_state(const ClothDesc* desc, int32_t B, int64_t total_nodes, const int64_t* node_cloth_start,
                             const float* x, const float* v, float* state, cudaStream_t s);
cudaError_t launch_get_state(const ClothDesc* desc, int32_t B, int64_t total_nodes, const int64_t* node_cloth_start,
                             const float* state, float* x, float* v, cudaStream_t s);
cudaError_t launch_fallback_check(const ClothDesc* desc, int B, int64_t max_nodes, int32_t* mode, float* resid,
                                  float* last, float bound, const float* net, float* dst, cudaStream_t s);
// Bounded-wait self-test (selftest.cu): a wait that cannot complete gives up
// after `polls` polls and sets kStatusTimeout.
cudaError_t launch_wait_timeout_selftest(int32_t* status, uint32_t polls, cudaStream_t s);
// Implicit plain step (implicit.cu): one linearised backward Euler step of
// h from `state` into `dst`; f_abi holds the explicit forces at `state`.
// blk[b]: the first of cloth b's blocks of implicit_block_nodes() nodes in
// a flat grid of n_blocks blocks over all cloths.
int implicit_grid_x(int64_t max_nodes);
int implicit_block_nodes();
cudaError_t launch_implicit_step(const ClothDesc* desc, const uint32_t* pinmask, int B, int64_t max_nodes,
                                 const int32_t* blk, int n_blocks, const float* state, const float* f_abi, float* dst,
                                 float* vecs, int64_t state_floats, float* part, float* scal, float h, int cg_iters,
                                 int32_t* status, cudaStream_t s);
cudaError_t launch_topology(const ClothDesc* desc, int32_t b, int32_t rows, int32_t cols, uint16_t* mask,
                            cudaStream_t s);

}  // namespace cloth
