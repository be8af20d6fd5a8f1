/*
 * libcloth — GB300 (sm_103a) C ABI for the regular-grid mass-spring cloth
 * and the physics-embedded CNN step of "A Physics-embedded Deep Learning
 * Framework for Cloth Simulation" (Zhao, arXiv 2403.12820).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an int status: CLOTH_OK (0) or a negative
 *    CLOTH_E* code; cloth_strerror() gives its text.  A CUDA failure returns
 *    CLOTH_ECUDA and cloth_last_cuda_error() gives the cudaError_t value
 *    (per calling thread).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that take a stream only enqueue work on it and return
 *    without synchronising, unless they say otherwise.
 *  - Pointers named d_* are device pointers, h_* host pointers.
 *  - Ownership: the caller allocates every device buffer, including the
 *    context workspace sized by cloth_workspace_size(); the library never
 *    allocates device memory.  A context owns only its host-side struct, a
 *    private capture stream and the CUDA graphs it caches; cloth_destroy()
 *    releases those.  The caller keeps the workspace alive until then.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Errors found on the device (non-finite state, bad index in a debug
 *    build) are OR-ed into a status word inside the workspace; read it with
 *    cloth_status().
 *
 * State layout at the ABI: the cloths of a batch are packed one after the
 * other; cloth b holds rows_b * cols_b nodes in row-major order, node
 * (r, c) at index r * cols_b + c, and each node three consecutive floats
 * (x, y, z).  Node (r, c) of cloth b rests at X = (c h_b, r h_b, 0).
 */
#ifndef CLOTH_H
#define CLOTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CLOTH_OK = 0,
    CLOTH_EINVAL = -1,       /* bad argument (NULL, size out of range, ...)   */
    CLOTH_ENOMEM = -2,       /* caller's workspace smaller than required      */
    CLOTH_ECUDA = -3,        /* a CUDA runtime call failed                    */
    CLOTH_ENONFINITE = -4,   /* non-finite value found in the state           */
    CLOTH_ETIMEOUT = -5,     /* a bounded device wait ran out                 */
    CLOTH_EUNSUPPORTED = -6  /* valid request this build does not implement  */
};

/* Bits of the device status word (cloth_status). */
enum {
    CLOTH_STATUS_NONFINITE = 1,   /* a step produced a non-finite x or v */
    CLOTH_STATUS_TIMEOUT = 2,     /* a bounded device wait ran out       */
    CLOTH_STATUS_BOUNDS = 4       /* reserved for index checks; no kernel of this library sets it */
};

/* Lattice of one cloth: rows x cols nodes, spacing h (m), node mass m (kg).
 * Sec. 3.1 (mass points joined by springs) and Sec. 4.1 (100 x 100 points). */
typedef struct {
    int32_t rows, cols;
    float spacing, mass;
} cloth_grid;

/* Material and loads of one cloth.
 *  k_struct, k_shear, k_bend: stiffness (N/m) of the springs to the 4
 *    cardinal neighbours, the 4 diagonal neighbours and the 4 nodes two
 *    apart in the cardinal directions — the 13-point stencil of Sec. 3.1,
 *    elastic force Eq. 1 with rest lengths h, sqrt(2) h, 2 h.
 *  mu_spring: spring-axis damping coefficient of Eq. 2.
 *  drag: air drag d of Eq. 4 (force -d v).
 *  pressure: p of Eq. 3, applied as (p/4) sum over the ordered cardinal
 *    pairs (E,N),(N,W),(W,S),(S,E) of x_ij1 x x_ij2 (a flat interior node
 *    receives p h^2 along +z).
 *  gravity: acceleration g of Eq. 4 (force m g). */
typedef struct {
    float k_struct, k_shear, k_bend, mu_spring, drag, pressure;
    float gravity[3];
} cloth_params;

/* Pinned nodes of one cloth (Sec. 3.1; the constraint operator C of Eq. 5
 * sets their velocity).  They move with `velocity` (m/s), the velocity of
 * the object they are attached to: zero holds them in place (the Dirichlet
 * case), anything else carries them along (a cloth part that moves with
 * another object).  `node` is a HOST array of `count` node indices
 * r * cols + c, read during cloth_create only. */
typedef struct {
    int32_t count;
    const int32_t* node;
    float velocity[3];
} cloth_pins;

/* Sphere obstacle (cloth-object intersection elimination, Sec. 3.1): after
 * each step a node inside the sphere is moved to the nearest point of its
 * surface.  friction < 0: the node stops (the ball of Sec. 3.2.2 that
 * absorbs the bounce and whose friction prevents relative motion).
 * friction >= 0: a Coulomb coefficient mu; with n the outward normal, the
 * approaching normal speed j = max(-v.n, 0) is absorbed, a separating
 * normal speed is kept, and the tangential speed loses min(|v_t|, mu j). */
typedef struct {
    float center[3];
    float radius;
    int32_t enabled;
    float friction;
} cloth_sphere;

typedef struct cloth_ctx cloth_ctx;

/* Bytes of device workspace a context for these B cloths needs (state
 * double buffer, descriptors, pin masks, work list, status word).
 * Returns CLOTH_EINVAL if B < 1 or a grid has rows or cols < 1. */
int cloth_workspace_size(int32_t B, const cloth_grid* grids, size_t* bytes);

/* Create a context for B cloths on the current CUDA device.
 *  grids, params: host arrays of B entries.  pins: host array of B entries
 *  or NULL (no pins).  spheres: host array of B entries or NULL.
 *  dt: time step of Eq. 5 (s).  d_workspace: device buffer of at least
 *  cloth_workspace_size() bytes, 256-byte aligned.
 * The workspace is initialised on `stream` (state zeroed: every cloth at
 * rest, zero velocity).  Returns CLOTH_EINVAL for a bad pin index or a
 * non-positive dt, spacing or mass; CLOTH_ENOMEM if `bytes` is too small. */
int cloth_create(cloth_ctx** out, int32_t B, const cloth_grid* grids, const cloth_params* params,
                 const cloth_pins* pins, const cloth_sphere* spheres, float dt,
                 void* d_workspace, size_t bytes, void* stream);

/* Load positions and velocities (packed ABI layout, device pointers, 3
 * floats per node, total_nodes = sum rows_b * cols_b).  d_v may be NULL
 * (zero velocity). */
int cloth_set_state(cloth_ctx* ctx, const float* d_x, const float* d_v, void* stream);

/* Store the current positions and velocities in the packed ABI layout.
 * Either pointer may be NULL to skip it. */
int cloth_get_state(cloth_ctx* ctx, float* d_x, float* d_v, void* stream);

/* Total force on every node at the current state — Eq. 1 + 2 (springs),
 * Eq. 3 (pressure) and Eq. 4 (gravity, drag) — packed like x. */
int cloth_forces(cloth_ctx* ctx, float* d_f, void* stream);

/* Advance every cloth `steps` plain steps (steps >= 0): the forces above,
 * then the semi-implicit Euler update of Eq. 5, v <- C(v + dt f / m),
 * x <- x + dt v, with pinned velocities set to their pins' velocity (zero
 * unless cloth_pins.velocity or cloth_set_boundary says otherwise), then
 * sphere contact.  One batched launch per step. */
int cloth_step_plain(cloth_ctx* ctx, int32_t steps, void* stream);

/* Rollout options.
 *  steps: number of steps to run.
 *  graph_chunk: steps per captured CUDA graph (rounded up to even; 0 =
 *    no graph, one launch per step).  The graph is captured on the
 *    context's private stream the first time a chunk size is used, cached
 *    in the context and replayed on `stream`.
 *  d_record / record_every: if d_record is not NULL, the positions after
 *    every `record_every`-th step are written to d_record in the packed ABI
 *    layout, one frame of 3 * total_nodes floats after another
 *    (steps / record_every frames).  Recording disables graphs. */
typedef struct {
    int32_t steps;
    int32_t graph_chunk;
    float* d_record;
    int32_t record_every;
} cloth_rollout_opts;

/* Plain-step rollout under the options above. */
int cloth_rollout_plain(cloth_ctx* ctx, const cloth_rollout_opts* opts, void* stream);

/* Memory of the Eq. 8 unroll (cloth_train_loss*): with k >= 1 only every
 * k-th unrolled state is kept, and the backward sweep recomputes the others
 * of a segment from its checkpoint when it reaches the segment: (S / k + k)
 * states instead of S + 1, about one more cell forward per unrolled step
 * (k near sqrt(S) minimises the memory).  k = 0 (the default) keeps every
 * state.  Loss and gradient are bitwise the same either way.  Query
 * cloth_train_workspace_size after this call.  CLOTH_EINVAL for k < 0. */
int cloth_set_train_segment(cloth_ctx* ctx, int32_t k);

/* Implicit plain step (Sec. 3.1: implicit integration is the stable choice
 * for large time steps; Sec. 5: the comparison for a larger-step cell):
 * `steps` linearised backward Euler steps of h = stride dt.  Per step, with
 * the elastic springs (Eq. 1) and the air drag (Eq. 4) implicit and the
 * rest (Eq. 2 damping, Eq. 3 pressure, gravity) explicit:
 *   (m + h d) dv - h^2 K dv = h f(x, v) + h^2 K v,  v' = C(v + dv),
 *   x' = x + h v', then sphere contact,
 * K the springs' stiffness matrix (per spring k [n n^T + max(0, 1 - L/l)
 * (I - n n^T)], n the unit spring vector, l its length), solved per cloth
 * by cg_iters conjugate-gradient iterations (matrix-free, pinned nodes
 * dv = pin_v - v).  d_work: cloth_implicit_workspace_size bytes, 256-byte
 * aligned.  Bitwise reproducible.  CLOTH_EINVAL for steps < 0, stride
 * outside 1..1000 or cg_iters < 0; CLOTH_ENOMEM for a short workspace;
 * CLOTH_EUNSUPPORTED for a cloth of 2^31 / 6 padded nodes or more. */
int cloth_implicit_workspace_size(const cloth_ctx* ctx, size_t* bytes);
int cloth_step_implicit(cloth_ctx* ctx, int32_t steps, int32_t stride, int32_t cg_iters, void* d_work, size_t bytes,
                        void* stream);

/* Larger-step network (Sec. 5: larger-step time integration with the
 * cell): from now on one network step (cloth_step_net, cloth_step_pcell,
 * cloth_rollout_net) advances k plain-step time steps, dt_net = k dt, in
 * the Euler update of Fig. 2; the plain step keeps dt.  The training loss
 * (cloth_train_loss*) unrolls with dt_net: its targets are then the
 * positions k, 2k, ... S k plain steps after the window start, and its
 * physics target is the mean acceleration of the k plain steps from the
 * window start, (v_k - v_0) / dt_net, less the start's pressure term.
 * k = 1 restores the plain time step.  In cloth_rollout_net a cloth on the
 * plain step (fallback) advances k plain steps per network step, and the
 * residual check compares the network step with k plain steps from the same
 * state; its workspace (cloth_net_rollout_workspace_size, to be queried
 * after this call) then holds a second scratch state.  CLOTH_EINVAL for k
 * outside 1..1000.  Synchronises `stream`. */
int cloth_set_net_stride(cloth_ctx* ctx, int32_t k, void* stream);

/* Boundary treatment of cloth b, selectable between steps (Sec. 3.2: BC
 * types are hard-encoded and selected at run time): the velocity its pinned
 * nodes move with (host array of 3 floats, as cloth_pins.velocity) and its
 * sphere's friction (as cloth_sphere.friction; ignored without a sphere).
 * Every step kernel reads them from the context's descriptors, so cached
 * graphs stay valid.  CLOTH_EINVAL for a bad b, a NULL pin_velocity or a
 * non-finite value.  Synchronises `stream`. */
int cloth_set_boundary(cloth_ctx* ctx, int32_t b, const float* pin_velocity, float sphere_friction, void* stream);

/* Launch shape of the plain step.  Every warp of the launch runs a
 * contiguous range of a work list of (cloth, 120-column strip, row segment)
 * units:
 *  seg_rows >= 4: strips cut into segments of that many rows, longest
 *    first, dealt round-robin to the warps (the default, with a segment
 *    length picked from the batch);
 *  seg_rows = -1: balanced ranges, the strips' rows cut into equal shares,
 *    one per warp;
 *  seg_rows = 0 keeps the current choice.
 * warps_per_sm (1..64) sets the warps of the launch to that many per SM;
 * -1 restores the default (one warp per segment, or for balanced ranges as
 * many warps as are resident at once); 0 keeps the current value.
 * Changes only speed, never results.  Cached graphs are dropped.
 * Synchronises `stream`. */
int cloth_set_launch(cloth_ctx* ctx, int32_t seg_rows, int32_t warps_per_sm, void* stream);

/* Launch-shape autotuner of the plain step.  For each of the n candidates
 * (seg_rows[i], warps_per_sm[i]), in cloth_set_launch's ranges (seg_rows
 * >= 4 or -1 for balanced ranges; warps_per_sm 1..64 or -1 for the
 * default), captures `steps` plain steps as one CUDA graph (as rollouts
 * replay them), replays it warmup + 1 times untimed and twice timed with
 * CUDA events on `stream`, and writes the mean microseconds per step to
 * us_out[i] (host array of n).  The steps read the current state
 * and write only the other state buffer: the state is unchanged.  The
 * fastest candidate is then applied as by cloth_set_launch and its index
 * written to *best (host).  CLOTH_EINVAL, before anything runs, for n < 1,
 * null arrays, warmup < 0, steps < 1 or a candidate out of range.  Cached
 * graphs are dropped.  Synchronises `stream`. */
int cloth_tune_launch(cloth_ctx* ctx, int32_t n, const int32_t* seg_rows, const int32_t* warps_per_sm,
                      int32_t warmup, int32_t steps, float* us_out, int32_t* best, void* stream);

/* Current launch shape: seg_rows (0 = balanced ranges), warps_per_sm (0 =
 * the default), number of work units. */
int cloth_get_launch(const cloth_ctx* ctx, int32_t* seg_rows, int32_t* warps_per_sm, int32_t* n_units);

/* Tile shapes of the fused network step of cloth_step_net /
 * cloth_rollout_net (Fig. 2) for networks of `precision`.  Choice v has
 * output tiles of rows[v] x cols[v] nodes on kinds[v]: 0 = the CUDA cores
 * (FP32), 1 = the tensor cores (tcgen05; for CLOTH_NET_FP32 each FP32 product
 * as three BF16 products, hi hi + hi lo + lo hi, of the operands split into a
 * high and a low BF16 part, with tanh and N + D in FP32).  FP32: two
 * tensor-core shapes (10 and 6 rows), then three CUDA-core shapes; BF16:
 * three tensor-core shapes (14, 10 and 6 rows).  Writes at most `capacity` entries to the host arrays and the
 * number of choices to *count; choice 0 is the default.  CLOTH_EINVAL for
 * another precision.  Host only. */
int cloth_net_tile_choices(int32_t precision, int32_t* rows, int32_t* cols, int32_t* kinds, int32_t capacity,
                           int32_t* count);

/* Select the tile shape of the precision's network step (a choice index;
 * else CLOTH_EINVAL).  Shapes of one kind give the same results, bit for bit
 * (each node's arithmetic does not depend on the tiling); the FP32 shapes of
 * the two kinds agree within the FP32 tolerance.  Cached network-rollout
 * graphs are dropped when it changes. */
int cloth_set_net_tile(cloth_ctx* ctx, int32_t precision, int32_t choice);
int cloth_get_net_tile(const cloth_ctx* ctx, int32_t precision, int32_t* choice);


/* Topology as the step kernels see it: for every node of cloth b, bit s of
 * d_mask[node] is set iff spring s exists (both ends in the grid), with s in
 * the order E, N, W, S, NE, NW, SW, SE, 2E, 2N, 2W, 2S (offsets (dr, dc):
 * (0,1) (1,0) (0,-1) (-1,0) (1,1) (1,-1) (-1,-1) (-1,1) (0,2) (2,0) (0,-2)
 * (-2,0)).  Sec. 3.1, 13-point stencil. */
int cloth_topology(cloth_ctx* ctx, int32_t b, uint16_t* d_mask, void* stream);

/* Synchronise `stream`, then read and return (in *h_status) the device
 * status word; with clear != 0 it is reset to 0 afterwards. */
int cloth_status(cloth_ctx* ctx, int32_t* h_status, int32_t clear, void* stream);

/* Self-test of the bounded waits: one warp waits `polls` polls on an
 * mbarrier that nothing completes, then gives up, sets
 * CLOTH_STATUS_TIMEOUT in the context's status word and returns (the path a
 * tensor-core wait that runs out takes).  The context stays usable.
 * CLOTH_EINVAL for polls < 1. */
int cloth_selftest_wait_timeout(cloth_ctx* ctx, int32_t polls, void* stream);

/* Number of cloths and total nodes of the context. */
int cloth_info(const cloth_ctx* ctx, int32_t* B, int64_t* total_nodes);

/* ------------------------------------------------------------------------
 * The physics-embedded CNN cell (Sec. 3.2, Eq. 6-7, Fig. 1) and the network
 * step of the framework (Fig. 2).
 *
 * The cell maps the displacement u = x - X and velocity v of every node to
 * an acceleration a (3 channels):
 *   zu = in_scale[0:3] u,  zv = in_scale[3:6] v
 *   phi1 = W1 (*) [zu; 0],  xi1 = W1 (*) [0; zv]       (Eq. 6, one kernel
 *   phi  = W2 (*) phi1,     xi  = W2 (*) xi1            for x and v)
 *   L = WL (*) phi + bL;  s = tanh(P phi);  N = WN s;  D = WD (xi . s)  (Eq. 7)
 *   a = out_scale (L + N + D)
 * with (*) a 3x3 cross-correlation with zero "same" padding, W1 6->32,
 * W2 32->32, WL 32->3, P 32->32 (1x1), WN, WD 32->3 (1x1).
 *
 * Weight blob (floats, this order): W1[32][6][3][3], W2[32][32][3][3],
 * WL[3][32][3][3], bL[3], P[32][32], WN[3][32], WD[3][32], in_scale[6],
 * out_scale[3] — CLOTH_NET_BLOB floats; gradients cover the first
 * CLOTH_NET_PARAMS (the scales are fixed).
 * ---------------------------------------------------------------------- */
#define CLOTH_NET_PARAMS 13027
#define CLOTH_NET_BLOB 13036

enum {
    CLOTH_NET_FP32 = 0,   /* FP32 CUDA-core arithmetic throughout            */
    CLOTH_NET_BF16 = 1    /* BF16 tensor-core channel contractions, FP32 accumulate */
};

typedef struct cloth_net cloth_net;

/* Device workspace of a network: the FP32 weights; the composite-trunk
 * operands of the network steps, repacked by net_create and
 * net_set_weights (the trunk of Eq. 6 with P and the linear branch of Eq. 7
 * folded into one 5x5 kernel, in BF16 for the tensor cores and FP32 for
 * the CUDA cores, and FP32 edge terms); and the per-block partial sums of
 * net_backward. */
int net_workspace_size(size_t* bytes);

/* Create a network on the current device from a HOST weight blob of
 * CLOTH_NET_BLOB floats.  precision: CLOTH_NET_FP32 or CLOTH_NET_BF16.
 * d_workspace: net_workspace_size() bytes, 256-byte aligned, owned by the
 * caller.  Returns CLOTH_EINVAL for a bad precision or a non-finite weight. */
int net_create(cloth_net** out, int32_t precision, const float* h_blob, void* d_workspace, size_t bytes,
               void* stream);

/* Replace the weights from a DEVICE blob of CLOTH_NET_BLOB floats (for
 * instance after an optimizer step); enqueued on `stream`. */
int net_set_weights(cloth_net* net, const float* d_blob, void* stream);

/* Copy the current weights (CLOTH_NET_BLOB floats) to a device buffer. */
int net_get_weights(const cloth_net* net, float* d_blob, void* stream);

/* Bytes of the activation buffer net_forward saves for net_backward, for
 * N images of H x W nodes (260 floats per node). */
int net_saved_size(int32_t N, int32_t H, int32_t W, size_t* bytes);

/* Forward of the cell on N images of H x W nodes, NCHW FP32:
 * d_z [N][6][H][W] (channels u_x u_y u_z v_x v_y v_z, u = x - X) ->
 * d_a [N][3][H][W].  If d_saved is not NULL (net_saved_size() bytes) the
 * activations needed by net_backward are stored there.  An FP32 network
 * runs on CUDA cores; a BF16 network runs its channel contractions on the
 * tensor cores (d_saved must then be NULL).  Sec. 3.2, Eq. 6-7. */
int net_forward(cloth_net* net, const float* d_z, float* d_a, int32_t N, int32_t H, int32_t W, float* d_saved,
                void* stream);

/* Backward of the cell (FP32 networks): given d_grad_a [N][3][H][W] =
 * dLoss/da at the forward's input d_z and its d_saved activations, ADDS
 * dLoss/dw to d_grad_w [CLOTH_NET_PARAMS] and, if d_grad_z is not NULL,
 * writes dLoss/dz [N][6][H][W].  d_saved is used as scratch and is no
 * longer valid afterwards.  Weight gradients are reduced in a fixed order
 * (bitwise reproducible).  Returns CLOTH_EUNSUPPORTED for a BF16 network. */
int net_backward(cloth_net* net, const float* d_z, float* d_saved, const float* d_grad_a, float* d_grad_z,
                 float* d_grad_w, int32_t N, int32_t H, int32_t W, void* stream);

/* net_forward_static — the FP32 cell forward for callers that cannot
 * allocate device memory on demand (for example a plug-in inside a host
 * application that reserves the GPU memory budget at start-up, or a
 * real-time frame loop where an allocation could stall a frame).  The paper
 * has no counterpart: this is a deployment variant of net_forward.
 *  d_blob: DEVICE weight blob of CLOTH_NET_BLOB floats (read only; no
 *    network handle needed).  d_z [N][6][H][W] in, d_a [N][3][H][W] out, as
 *    for net_forward.
 * The trunk's layer outputs live in one static device array inside the
 * library (CLOTH_NET_STATIC_MAX_NODES nodes, 8 MiB, held by every GPU that
 * loads the library until exit); nothing is allocated.  Returns
 * CLOTH_EINVAL when N * H * W exceeds CLOTH_NET_STATIC_MAX_NODES.  The first
 * call on a device looks up the array's device address and sets kernel
 * attributes; make that first call before any stream capture.  Both are
 * kept until exit, so a cudaDeviceReset after the first call on a device is
 * not supported.  All calls on a device share the array: calls whose work
 * overlaps on the GPU race.  On CLOTH_ECUDA, cloth_last_cuda_error gives the
 * cudaError_t. */
#define CLOTH_NET_STATIC_MAX_NODES 16384
int net_forward_static(const float* d_blob, const float* d_z, float* d_a, int32_t N, int32_t H, int32_t W,
                       void* stream);

/* Release the network's host resources. */
void net_destroy(cloth_net* net);

/* Device workspace cloth_step_net needs for this context and network
 * precision (the list of output tiles of its fused step kernel). */
int cloth_net_workspace_size(const cloth_ctx* ctx, int32_t precision, size_t* bytes);

/* Advance every cloth `steps` network steps (Fig. 2): a = cell(u, v), then
 * v <- C(v + dt (a + f_p / m)), x <- x + dt v with the pressure f_p of Eq. 3
 * and the pins hard-encoded outside the network, then sphere contact.  One
 * fused kernel per step for the whole batch: the tensor-core kernel for a
 * BF16 network, the CUDA-core kernel for an FP32 one; both evaluate the
 * trunk through the composite kernel (exact algebra, FP32 edge terms on the
 * cloth's outermost ring), so results differ from net_forward's layered
 * evaluation only by rounding.  d_work: cloth_net_workspace_size() bytes
 * (the tile list). */
int cloth_step_net(cloth_ctx* ctx, const cloth_net* net, int32_t steps, void* d_work, size_t bytes, void* stream);

/* Launch-shape tuner of the network step: runs `warmup` untimed and `steps`
 * timed network steps of `net` in every tile shape of its precision (CUDA
 * events on `stream`; each step reads the current state and writes the
 * other buffer, so the state does not move), writes microseconds per step
 * to us_out[v] (host, one per choice, in the order of
 * cloth_net_tile_choices), selects the fastest and writes its index to
 * *best (host).  d_work is a device workspace of
 * cloth_net_workspace_size(ctx, precision) bytes.  Cached graphs are
 * dropped.  Synchronises `stream`. */
int cloth_tune_net(cloth_ctx* ctx, const cloth_net* net, int32_t warmup, int32_t steps, float* us_out, int32_t* best,
                   void* d_work, size_t bytes, void* stream);

/* Network rollout with the plain step as fallback and judge (Fig. 2: the
 * framework couples the network with the physics-based simulator).
 *  steps: steps to run.  check_every: every check_every-th step (0 = never)
 *    both steps start from the same state; cloth b's residual r_b is the
 *    largest |x_net - x_plain| over its nodes (m), and if r_b exceeds
 *    residual_bound the cloth is switched to the plain step for the rest of
 *    the rollout (the switch persists until cloth_reset_modes) and takes the
 *    plain result of that step.
 *  graph_chunk: steps per captured CUDA graph (rounded up to a whole number
 *    of check periods and an even count; 0 = no graph). */
typedef struct {
    int32_t steps;
    int32_t check_every;
    float residual_bound;
    int32_t graph_chunk;
} cloth_net_rollout_opts;

/* Workspace of cloth_rollout_net (tile list and one scratch state). */
int cloth_net_rollout_workspace_size(const cloth_ctx* ctx, int32_t precision, size_t* bytes);

/* Network rollout under the options above, for either precision: the
 * network steps are the fused kernels of cloth_step_net. */
int cloth_rollout_net(cloth_ctx* ctx, const cloth_net* net, const cloth_net_rollout_opts* opts, void* d_work,
                      size_t bytes, void* stream);

/* Per-cloth step mode (0 = network, 1 = plain after a failed check) and the
 * residual of the cloth's last check (m; for a switched cloth, the one that
 * switched it), copied to device arrays of B entries; either pointer may be
 * NULL.  Stream-ordered. */
int cloth_modes(cloth_ctx* ctx, int32_t* d_mode, float* d_residual, void* stream);

/* Switch every cloth back to the network step. */
int cloth_reset_modes(cloth_ctx* ctx, void* stream);

/* ------------------------------------------------------------------------
 * The physics-embedded cell read literally (Sec. 3.2, Eq. 6-7, Fig. 1).
 *
 * Per coordinate k (the same 2D kernels act on x, y and z: isotropy) and
 * node i, over the 12 stencil neighbours j_c that exist (channel c is the
 * frozen difference filter of one neighbour; order E, W, N, S, NE, NW, SE,
 * SW, E2, W2, N2, S2 with N = row + 1, E = column + 1, and the "2" taps two
 * apart, a dilation-2 kernel):
 *   phi_c = x_jc - x_i,  xi_c = v_jc - v_i,
 *   s_c = phi_c / sqrt(1 + alpha phi_c^2)          (ISRU activation)
 *   a_k = b_L[k] + sum_c (w_L[c] phi_c + w_N[c] s_c + w_D[c] xi_c s_c)
 * Weight blob, device, CLOTH_PCELL_BLOB floats:
 *   w_L[12], w_N[12], w_D[12], b_L[3], alpha.
 * The blob is read on every call; the caller keeps it finite.  The
 * workspace holds the tile list: size from cloth_pcell_workspace_size,
 * 256-byte aligned. */
#define CLOTH_PCELL_BLOB 40

int cloth_pcell_workspace_size(const cloth_ctx* ctx, size_t* bytes);

/* The cell's output a at the current state into d_a (packed [node][3], the
 * order of cloth_get_state).  State unchanged.  Stream-ordered. */
int cloth_pcell_accel(cloth_ctx* ctx, const float* d_w, float* d_a, void* d_work, size_t bytes, void* stream);

/* `steps` network steps of Fig. 2 with the literal cell: a + (pressure of
 * Eq. 3) / m drives Eq. 5 with the pins and sphere contact of the context.
 * Stream-ordered; a non-finite position sets CLOTH_STATUS_NONFINITE. */
int cloth_step_pcell(cloth_ctx* ctx, const float* d_w, int32_t steps, void* d_work, size_t bytes, void* stream);

/* ------------------------------------------------------------------------
 * Training (Sec. 3.2.1, Eq. 8; Table 1)
 * ---------------------------------------------------------------------- */

/* Device workspace of cloth_train_loss for this context and unroll length. */
int cloth_train_workspace_size(const cloth_ctx* ctx, int32_t S, size_t* bytes);

/* Loss of Eq. 8 and its gradient for a batch of training windows.
 * The context holds one window per cloth (all cloths of one size, each
 * with its own pins and pressure); its current state is the window start
 * (x_k, v_k).  d_targets [S][total_nodes][3] (packed ABI layout) holds the
 * recorded positions x_{k+1} .. x_{k+S}.  Per window:
 *   L = alpha * mean_free(((a_net(x_k, v_k) - a_true) / g_norm)^2)
 *     + (1 - alpha) / S * sum_{s=1..S} mean_free(((x_hat_{k+s} - x_{k+s}) / h)^2)
 * where a_true = (Eq. 1 + 2 + 4 force) / m at the window start (the plain
 * step's acceleration without the pressure, which the network step adds
 * itself), x_hat is the S-step network rollout of Fig. 2 (pressure and pins
 * hard-encoded, no sphere), means run over the free (unpinned) nodes and
 * their 3 components, and h is the cloth's spacing.  Writes the batch mean
 * of L to d_loss (1 device float) and ADDS its gradient with respect to the
 * CLOTH_NET_PARAMS weights to d_grad_w.  The gradient is the exact adjoint
 * (net_backward through every step, the Euler update, pins and pressure);
 * each step's activations are recomputed during the backward sweep (step
 * checkpointing).  d_grad_w may be NULL: the loss alone, without the
 * backward sweep (the objective of the differential-evolution pre-process
 * of Sec. 3.2.1).  The context state is left unchanged.  FP32 networks only
 * (CLOTH_EUNSUPPORTED otherwise); CLOTH_EINVAL if the cloths differ in size. */
int cloth_train_loss(cloth_ctx* ctx, cloth_net* net, int32_t S, const float* d_targets, float alpha, float g_norm,
                     float* d_loss, float* d_grad_w, void* d_work, size_t bytes, void* stream);

/* The same loss and gradient with the literal cell (d_w: CLOTH_PCELL_BLOB
 * floats, see cloth_pcell_accel) as the network: ADDS the gradient with
 * respect to its 39 trainable entries to d_grad_w[0..38] (alpha, entry 39,
 * is fixed and left alone); d_grad_w may be NULL (the loss alone).  Same
 * workspace (cloth_train_workspace_size); the parameter gradient is summed
 * in a fixed order (bitwise reproducible). */
int cloth_train_loss_pcell(cloth_ctx* ctx, const float* d_w, int32_t S, const float* d_targets, float alpha,
                           float g_norm, float* d_loss, float* d_grad_w, void* d_work, size_t bytes, void* stream);

/* One Adam update (Table 1's optimizer) of n parameters in place:
 * m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
 * w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * All pointers are device arrays of n floats; t >= 1 is the step count. */
int net_adam_step(float* d_w, const float* d_grad, float* d_m, float* d_v, int32_t n, int32_t t, float lr,
                  float beta1, float beta2, float eps, void* stream);

/* The same update on the entries whose byte of d_mask (device, n bytes) is
 * non-zero; the others keep w, m and v.  Branch-wise fine-tuning with the
 * other branches frozen (Sec. 5): the mask selects the trainable groups. */
int net_adam_step_masked(float* d_w, const float* d_grad, float* d_m, float* d_v, const uint8_t* d_mask, int32_t n,
                         int32_t t, float lr, float beta1, float beta2, float eps, void* stream);

/* Release the context's host resources (graphs, capture stream). */
void cloth_destroy(cloth_ctx* ctx);

const char* cloth_strerror(int code);
int cloth_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CLOTH_H */
