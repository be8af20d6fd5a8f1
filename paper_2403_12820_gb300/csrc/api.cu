// Host implementation of the cloth context entry points of include/cloth.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/cloth.h"
#include "cloth_internal.cuh"
#include "net_internal.cuh"
#include "train_internal.cuh"

using namespace cloth;

namespace {

thread_local int g_last_cuda = 0;

constexpr int kMinSegRows = 4;       // smallest row segment the work list may use
constexpr int kMaxWarps = 1 << 16;   // bound on the warps of one plain-step launch
constexpr int kMaxNetStride = 1000;  // bound on the plain steps one network step may span
constexpr size_t kAlign = 256;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int64_t pitch_of(int cols) { return (int64_t)((cols + kPitchAlign - 1) / kPitchAlign) * kPitchAlign; }

// Work units of `seg_rows`-row segments of `strip`-column strips (the plain
// kernel's kStrip by default; the narrower strip bounds the layout).
int64_t units_for(const cloth_grid* g, int B, int seg_rows, int strip = kStrip)
{
    int64_t n = 0;
    for (int b = 0; b < B; ++b)
        n += (int64_t)((g[b].cols + strip - 1) / strip) * ((g[b].rows + seg_rows - 1) / seg_rows);
    return n;
}

struct Layout {
    size_t desc, units, warp_first, pins, pin_list, state[2], status, ctl, total;
    int64_t state_floats, pin_words, max_units, pin_list_cap;
};

Layout make_layout(int B, const cloth_grid* g)
{
    Layout L{};
    int64_t floats = 0, words = 0;
    for (int b = 0; b < B; ++b) {
        const int64_t pitch = pitch_of(g[b].cols);
        floats += align_up((size_t)(6 * g[b].rows * pitch), kAlign / sizeof(float));
        words += (int64_t)g[b].rows * ((pitch + 31) / 32);
    }
    L.state_floats = floats;
    L.pin_words = words;
    // fixed segments split every strip; balanced ranges split each strip at
    // most once per warp
    L.max_units = std::max<int64_t>(units_for(g, B, kMinSegRows), units_for(g, B, 1 << 30) + kMaxWarps);
    size_t off = 0;
    L.desc = off;     off = align_up(off + sizeof(ClothDesc) * B, kAlign);
    L.units = off;    off = align_up(off + sizeof(WorkUnit) * L.max_units, kAlign);
    L.warp_first = off; off = align_up(off + sizeof(int32_t) * (kMaxWarps + 1), kAlign);
    L.pins = off;     off = align_up(off + sizeof(uint32_t) * words, kAlign);
    // the pinned nodes as (cloth, node) pairs: room for one per pin word
    // (one node in 32; more pins than that are set from the mask instead)
    L.pin_list_cap = std::max<int64_t>(words, 64);
    L.pin_list = off; off = align_up(off + sizeof(int2) * L.pin_list_cap, kAlign);
    L.state[0] = off; off = align_up(off + sizeof(float) * floats, kAlign);
    L.state[1] = off; off = align_up(off + sizeof(float) * floats, kAlign);
    L.status = off;   off = align_up(off + 64, kAlign);
    L.ctl = off;      off = align_up(off + 12 * (size_t)B, kAlign);   // modes, residuals, last residuals
    L.total = off;
    return L;
}

bool grids_ok(int32_t B, const cloth_grid* g)
{
    if (B < 1 || B > 65535 || !g) return false;
    for (int b = 0; b < B; ++b)
        if (g[b].rows < 1 || g[b].cols < 1 || g[b].rows > (1 << 20) || g[b].cols > (1 << 20)) return false;
    return true;
}

int cuda_fail(cudaError_t e)
{
    g_last_cuda = (int)e;
    return CLOTH_ECUDA;
}

// Cloths of one size, stepped by the network as one batch of images.

#define CK(expr)                                 \
    do {                                         \
        cudaError_t e__ = (expr);                \
        if (e__ != cudaSuccess) return cuda_fail(e__); \
    } while (0)

}  // namespace

struct cloth_ctx {
    int32_t B = 0;
    int64_t total_nodes = 0, max_nodes = 0;
    bool damp = false;
    char* ws = nullptr;
    Layout L{};
    std::vector<ClothDesc> desc;
    std::vector<cloth_grid> grids;
    int cur = 0;                       // state buffer holding the current state
    int seg_rows = 16;
    int n_units = 0;
    int n_warps = 0;                   // warps of one plain-step launch that have work
    int grid = 0, block = 128;
    int warps_per_sm = 0;              // 0: the plain-step kernel's occupancy
    int net_stride = 1;                // plain steps one network step spans
    int fp32_tile = 0;                 // tile shape of the FP32 network step (a choice of tile_shape)
    int bf16_tile = 0;                 // tile shape of the BF16 network step (a choice of tile_shape)
    int train_seg = 0;                 // Eq. 8 unroll: keep every train_seg-th state (0: all)
    int sm_count = 0;
    cudaStream_t cap = nullptr;        // private stream for graph capture
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (chunk, start buffer) -> graph
    // checked network rollouts: (network, its workspace, precision, rollout
    // workspace and size, chunk, check period, residual bound bits, start
    // buffer) -> graph
    using NetGraphKey = std::tuple<const void*, const void*, int, const void*, size_t, int, int, uint32_t, int>;
    std::map<NetGraphKey, cudaGraphExec_t> net_graphs;
    std::vector<int64_t> free_nodes;   // nodes per cloth that are not pinned
    int32_t n_pins = 0;                // entries of the pin list; -1: pins set from the mask
    std::vector<int32_t> impl_blk;     // implicit step: first block of each cloth, then the total
    const void* lists_written = nullptr;   // step workspace holding current cloth lists
    int lists_kind = -1;                   // which list it holds (network precision, FP32 tile shape)

    ClothDesc* d_desc() const { return reinterpret_cast<ClothDesc*>(ws + L.desc); }
    WorkUnit* d_units() const { return reinterpret_cast<WorkUnit*>(ws + L.units); }
    int32_t* d_warp_first() const { return reinterpret_cast<int32_t*>(ws + L.warp_first); }
    uint32_t* d_pins() const { return reinterpret_cast<uint32_t*>(ws + L.pins); }
    int2* d_pin_list() const { return reinterpret_cast<int2*>(ws + L.pin_list); }
    float* d_state(int k) const { return reinterpret_cast<float*>(ws + L.state[k]); }
    int32_t* d_status() const { return reinterpret_cast<int32_t*>(ws + L.status); }
    int32_t* d_mode() const { return reinterpret_cast<int32_t*>(ws + L.ctl); }
    float* d_resid() const { return reinterpret_cast<float*>(ws + L.ctl) + B; }
    float* d_last() const { return reinterpret_cast<float*>(ws + L.ctl) + 2 * B; }
};

namespace {

// Forget every cached rollout graph (the launch shape or the stride changed,
// or the context goes away).
void drop_graphs(cloth_ctx* c)
{
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    for (auto& kv : c->net_graphs) cudaGraphExecDestroy(kv.second);
    c->net_graphs.clear();
}

// Build and upload the work list of the plain step; every warp of the
// launch runs a contiguous range of it.
//  seg_rows > 0 (default: picked by pick_seg_rows): strips cut into
//    segments of `seg_rows` rows, longest first, dealt round-robin to the
//    warps.  By default there is one warp per segment: the blocks beyond
//    those resident start as earlier ones finish, which balances the tail,
//    and the warps of a block take horizontally adjacent strips of the same
//    rows (contiguous memory).
//  seg_rows = 0: balanced ranges.  The strips' rows, laid end to end, are
//    cut into equal shares, one per warp (by default as many as are resident
//    at once), so every warp marches the same number of rows (+- 1); a share
//    that spans two strips restarts its window once.
int set_work(cloth_ctx* c, int seg_rows, cudaStream_t s)
{
    const int warps_per_block = c->block / 32;
    const int strip = c->damp ? kStripDamp : kStrip;
    int wps = c->warps_per_sm;
    if (wps <= 0 && seg_rows <= 0) wps = std::max(1, plain_step_blocks_per_sm(c->damp, c->block)) * warps_per_block;
    const int W = wps > 0 ? std::max(1, std::min(kMaxWarps, c->sm_count * wps)) : kMaxWarps;
    std::vector<WorkUnit> u;
    std::vector<int32_t> first;
    if (seg_rows > 0) {
        seg_rows = std::max(seg_rows, kMinSegRows);
        std::vector<WorkUnit> all;
        for (int b = 0; b < c->B; ++b) {
            const int rows = c->grids[b].rows, cols = c->grids[b].cols;
            for (int r0 = 0; r0 < rows; r0 += seg_rows)
                for (int c0 = 0; c0 < cols; c0 += strip) all.push_back(WorkUnit{b, c0, r0, std::min(rows, r0 + seg_rows)});
        }
        std::stable_sort(all.begin(), all.end(),
                         [](const WorkUnit& a, const WorkUnit& b) { return (a.r1 - a.r0) > (b.r1 - b.r0); });
        const int nw = std::min<int>(W, (int)all.size());
        for (int w = 0; w < nw; ++w) {
            first.push_back((int32_t)u.size());
            for (size_t i = (size_t)w; i < all.size(); i += (size_t)nw) u.push_back(all[i]);
        }
    } else {
        int64_t total = 0;
        for (int b = 0; b < c->B; ++b)
            total += (int64_t)c->grids[b].rows * ((c->grids[b].cols + strip - 1) / strip);
        const int64_t q = std::max<int64_t>(1, (total + W - 1) / W);   // rows per warp
        int64_t pos = 0;
        for (int b = 0; b < c->B; ++b) {
            const int rows = c->grids[b].rows, cols = c->grids[b].cols;
            for (int c0 = 0; c0 < cols; c0 += strip)
                for (int r = 0; r < rows;) {
                    const int64_t w = pos / q;
                    const int take = (int)std::min<int64_t>(rows - r, (w + 1) * q - pos);
                    while ((int64_t)first.size() <= w) first.push_back((int32_t)u.size());
                    u.push_back(WorkUnit{b, c0, r, r + take});
                    r += take;
                    pos += take;
                }
        }
    }
    first.push_back((int32_t)u.size());
    if ((int64_t)u.size() > c->L.max_units || (int)first.size() - 1 > kMaxWarps) return CLOTH_EINVAL;
    CK(cudaMemcpyAsync(c->d_units(), u.data(), sizeof(WorkUnit) * u.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_warp_first(), first.data(), sizeof(int32_t) * first.size(), cudaMemcpyHostToDevice, s));
    c->seg_rows = seg_rows > 0 ? seg_rows : 0;
    c->n_units = (int)u.size();
    c->n_warps = (int)first.size() - 1;
    c->grid = std::max(1, (c->n_warps + warps_per_block - 1) / warps_per_block);
    // the host vectors go out of scope: the copies must be done
    CK(cudaStreamSynchronize(s));
    return CLOTH_OK;
}

int pick_seg_rows(const cloth_ctx* c)
{
    // enough segments to cover every SM a dozen times, but long enough that
    // the 2 warm-up rows stay a small fraction
    const int64_t target = (int64_t)c->sm_count * 12;
    for (int R : {64, 32, 16, 8})
        if (units_for(c->grids.data(), c->B, R, c->damp ? kStripDamp : kStrip) >= target) return R;
    return 8;
}

// Plain step from src into dst; with `mode`, only cloths in plain mode.
int launch_plain(cloth_ctx* c, const float* src, float* dst, const int32_t* mode, cudaStream_t s)
{
    StepArgs a{};
    a.desc = c->d_desc();
    a.units = c->d_units();
    a.warp_first = c->d_warp_first();
    a.n_warps = c->n_warps;
    a.src = src;
    a.dst = dst;
    a.pinmask = c->d_pins();
    a.status = c->d_status();
    a.mode = mode;
    a.pin_list = c->d_pin_list();
    a.n_pins = c->n_pins;
    a.n_cloths = c->B;
    if (c->damp) CK(launch_plain_step_damp(a, false, c->grid, c->block, s));
    else CK(launch_plain_step(a, false, c->grid, c->block, s));
    return CLOTH_OK;
}

int launch_step(cloth_ctx* c, bool forces_only, float* force_out, cudaStream_t s)
{
    StepArgs a{};
    a.desc = c->d_desc();
    a.units = c->d_units();
    a.warp_first = c->d_warp_first();
    a.n_warps = c->n_warps;
    a.src = c->d_state(c->cur);
    a.dst = c->d_state(c->cur ^ 1);
    a.pinmask = c->d_pins();
    a.force_out = force_out;
    a.status = c->d_status();
    a.pin_list = c->d_pin_list();
    a.n_pins = c->n_pins;
    a.n_cloths = c->B;
    if (c->damp) CK(launch_plain_step_damp(a, forces_only, c->grid, c->block, s));
    else CK(launch_plain_step(a, forces_only, c->grid, c->block, s));
    if (!forces_only) c->cur ^= 1;
    return CLOTH_OK;
}

// Tiles (cloth, y0, x0, -) of R x WO output nodes over every cloth.
std::vector<int4> net_tiles(const cloth_ctx* c, int R, int WO)
{
    std::vector<int4> t;
    for (int b = 0; b < c->B; ++b)
        for (int y0 = 0; y0 < c->grids[b].rows; y0 += R)
            for (int x0 = 0; x0 < c->grids[b].cols; x0 += WO) t.push_back(make_int4(b, y0, x0, 0));
    return t;
}
// of the fused tensor-core (BF16) and CUDA-core (FP32) network steps
// Tile shapes of a precision's fused step: FP32 choice v < net_tc_split_variants()
// is the tensor-core kernel with three BF16 products per term in shape v (the
// default, the faster kind), the next ones the CUDA-core kernel in shape
// v - net_tc_split_variants(); BF16 choice v the tensor-core kernel in shape v.
int tile_choices(int precision)
{
    return precision == CLOTH_NET_BF16 ? net_tc_variants() : net_tc_split_variants() + net_comp_variants();
}
bool fp32_split(int v) { return v < net_tc_split_variants(); }
int fp32_comp(int v) { return v - net_tc_split_variants(); }
void tile_shape(int precision, int v, int* rows, int* cols, int* kind)
{
    if (precision == CLOTH_NET_BF16) {
        *rows = net_tc_variant_rows(v); *cols = net_tc_tile_cols(); *kind = 1;
    } else if (fp32_split(v)) {
        *rows = net_tc_split_rows(v); *cols = net_tc_tile_cols(); *kind = 1;
    } else {
        *rows = net_comp_tile_rows(); *cols = net_comp_variant_cols(fp32_comp(v)); *kind = 0;
    }
}
std::vector<int4> shape_tiles(const cloth_ctx* c, int precision, int v)
{
    int rows, cols, kind;
    tile_shape(precision, v, &rows, &cols, &kind);
    return net_tiles(c, rows, cols);
}
int& tile_variant(cloth_ctx* c, int precision) { return precision == CLOTH_NET_BF16 ? c->bf16_tile : c->fp32_tile; }
int tile_variant(const cloth_ctx* c, int precision) { return precision == CLOTH_NET_BF16 ? c->bf16_tile : c->fp32_tile; }
std::vector<int4> net_step_tiles(const cloth_ctx* c, int precision)
{
    return shape_tiles(c, precision, tile_variant(c, precision));
}
// kind of a network's tile list (what the workspace holds)
int list_kind(const cloth_ctx* c, const cloth_net* net)
{
    return (net->precision == CLOTH_NET_BF16 ? 100 : 10) + tile_variant(c, net->precision);
}

// One fused network step over the tile list, in the context's tile shape for
// the network's precision: the tensor-core kernel (one CTA per SM) for a
// BF16 network or the FP32 three-term shape, else the FP32 composite kernel
// on the CUDA cores (as many blocks as are resident).  `mode` restricts it
// to the cloths in network mode.
int launch_net_step(const cloth_ctx* c, const cloth_net* net, const int4* d_tiles, int n_tiles, const float* src,
                    float* dst, const int32_t* mode, cudaStream_t s)
{
    const bool bf16 = net->precision == CLOTH_NET_BF16;
    if (bf16 || fp32_split(c->fp32_tile))
        CK(launch_net_tc_step(bf16 ? c->bf16_tile : c->fp32_tile, !bf16, net->d_pack(), net->d_w(), c->d_desc(),
                              d_tiles, n_tiles, src, dst, c->d_pins(), c->d_status(), std::min(n_tiles, c->sm_count),
                              s, mode));
    else
        CK(launch_net_comp_step(fp32_comp(c->fp32_tile), net->d_w(), net->d_comp(), net->d_edge(), c->d_desc(),
                                d_tiles, n_tiles, src, dst, c->d_pins(), c->d_status(),
                                std::min(n_tiles, net_comp_blocks_per_sm(fp32_comp(c->fp32_tile)) * c->sm_count), s,
                                mode));
    return CLOTH_OK;
}

// The network's tile list in the workspace (uploaded once per workspace and precision).
int net_tile_list(cloth_ctx* c, const cloth_net* net, void* d_work, size_t bytes, int* n_tiles, cudaStream_t s)
{
    const std::vector<int4> tiles = net_step_tiles(c, net->precision);
    if (bytes < sizeof(int4) * tiles.size()) return CLOTH_ENOMEM;
    if (c->lists_written != d_work || c->lists_kind != list_kind(c, net)) {
        CK(cudaMemcpyAsync(d_work, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        c->lists_written = d_work;
        c->lists_kind = list_kind(c, net);
    }
    *n_tiles = (int)tiles.size();
    return CLOTH_OK;
}

int step_net_fused(cloth_ctx* c, const cloth_net* net, int32_t steps, void* d_work, size_t bytes, cudaStream_t s)
{
    int n_tiles = 0;
    const int rc = net_tile_list(c, net, d_work, bytes, &n_tiles, s);
    if (rc) return rc;
    for (int st = 0; st < steps; ++st) {
        const int r = launch_net_step(c, net, static_cast<const int4*>(d_work), n_tiles, c->d_state(c->cur),
                                      c->d_state(c->cur ^ 1), nullptr, s);
        if (r) return r;
        c->cur ^= 1;
    }
    return CLOTH_OK;
}

// Workspace of cloth_train_loss (float offsets).
struct TrainWs {
    size_t z, a, at, ga0, gu, gv, ga, gfp, ge, gn, gz, saved, fabi, coef, part, ppart, kstate, total;
};
TrainWs train_ws(const cloth_ctx* c, int S)
{
    const int64_t B = c->B, HW = (int64_t)c->grids[0].rows * c->grids[0].cols, n3 = B * 3 * HW;
    TrainWs w{};
    size_t off = 0;
    auto take = [&](size_t floats) { const size_t o = off; off = align_up(off + floats, kAlign / sizeof(float)); return o; };
    // unrolled states kept: all S + 1, or with segments of k the checkpoints
    // t = 0, k, 2k, ... and one segment's k - 1 others
    const int k = c->train_seg;
    w.z = take((size_t)(k > 0 ? S / k + k : S + 1) * B * 6 * HW);
    w.a = take(n3); w.at = take(n3); w.ga0 = take(n3); w.gu = take(n3); w.gv = take(n3);
    w.ga = take(n3); w.gfp = take(n3); w.ge = take(n3); w.gn = take(n3);
    w.gz = take((size_t)B * 6 * HW);
    w.saved = take((size_t)kSavedPerNode * B * HW);
    w.fabi = take((size_t)3 * c->total_nodes);
    w.coef = take((size_t)2 * B);
    w.part = take((size_t)(S + 1) * train_blocks(c->grids[0].rows, c->grids[0].cols, c->B));
    w.ppart = take((size_t)40 * pcell_train_blocks(c->grids[0].rows, c->grids[0].cols, c->B));
    w.kstate = take((size_t)c->L.state_floats);   // plain steps of a stride > 1 (physics target)
    w.total = off * sizeof(float);
    return w;
}

bool same_size(const cloth_ctx* c)
{
    for (int b = 1; b < c->B; ++b)
        if (c->grids[b].rows != c->grids[0].rows || c->grids[b].cols != c->grids[0].cols) return false;
    return true;
}

}  // namespace

extern "C" {

int cloth_train_workspace_size(const cloth_ctx* c, int32_t S, size_t* bytes)
{
    if (!c || !bytes || S < 1 || !same_size(c)) return CLOTH_EINVAL;
    *bytes = train_ws(c, S).total;
    return CLOTH_OK;
}

}  // extern "C"

namespace {

// Eq. 8 for the windows held by the context, with the cell given by
// `forward(z_t, a)` (a = cell(z_t)) and `backward(z_t, ga, gz)` (gz = dL/dz_t
// through the cell, the parameter gradient added to the caller's grad_w).
template <class Fwd, class Bwd>
int train_loss_impl(cloth_ctx* c, int32_t S, const float* d_targets, float alpha, float g_norm, float* d_loss,
                    void* d_work, size_t bytes, cudaStream_t s, Fwd forward, Bwd backward, bool with_grad)
{
    if (!d_targets || !d_loss || !d_work || S < 1 || !same_size(c)) return CLOTH_EINVAL;
    if (!(alpha >= 0.f && alpha <= 1.f) || !(g_norm > 0.f)) return CLOTH_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_work) % kAlign) return CLOTH_EINVAL;
    const TrainWs L = train_ws(c, S);
    if (bytes < L.total) return CLOTH_ENOMEM;
    const int B = c->B, H = c->grids[0].rows, W = c->grids[0].cols;
    const int64_t HW = (int64_t)H * W, NHW = (int64_t)B * HW;
    float* ws = static_cast<float*>(d_work);
    float* Z = ws + L.z;
    // state t of the unroll: every state is kept (train_seg 0), or the
    // checkpoints t = 0, k, 2k, ... and, for the other t, the slot of its
    // place in the segment (one segment at a time)
    const int k = c->train_seg;
    const int n_ck = k > 0 ? S / k + 1 : S + 1;
    auto Zt = [&](int t) {
        const size_t slot = (k == 0 || t % k == 0) ? (size_t)(k ? t / k : t) : (size_t)(n_ck + t % k - 1);
        return Z + slot * B * 6 * HW;
    };
    float *A = ws + L.a, *AT = ws + L.at, *GA0 = ws + L.ga0, *GU = ws + L.gu, *GV = ws + L.gv;
    float *GA = ws + L.ga, *GFP = ws + L.gfp, *GE = ws + L.ge, *GN = ws + L.gn, *GZ = ws + L.gz;
    float *FABI = ws + L.fabi, *COEF = ws + L.coef, *PART = ws + L.part;
    const int blocks = train_blocks(H, W, B);
    const ClothDesc* D = c->d_desc();
    const uint32_t* P = c->d_pins();

    // per-window weights of the two terms (1/B: batch mean)
    std::vector<float> coef(2 * B);
    for (int b = 0; b < B; ++b) {
        const double cnt = 3.0 * (double)std::max<int64_t>(c->free_nodes[b], 1);
        const double h = c->desc[b].h;
        coef[b] = (float)(alpha / (cnt * (double)g_norm * g_norm * B));
        coef[B + b] = (float)((1.0 - alpha) / ((double)S * cnt * h * h * B));
    }
    CK(cudaMemcpyAsync(COEF, coef.data(), sizeof(float) * 2 * B, cudaMemcpyHostToDevice, s));

    // targets of the physics term: the plain step's acceleration without
    // pressure; for a network stride k > 1 the mean acceleration of k plain
    // steps from the window start (ping-pong between the spare state buffer
    // and the workspace; the current state is not touched)
    CK(launch_state_to_z(D, c->d_state(c->cur), Zt(0), B, H, W, s));
    if (c->net_stride == 1) {
        const int rc = launch_step(c, true, FABI, s);
        if (rc) return rc;
        CK(launch_a_true(D, FABI, Zt(0), AT, B, H, W, s));
    } else {
        float* bufs[2] = {c->d_state(c->cur ^ 1), ws + L.kstate};
        const float* from = c->d_state(c->cur);
        for (int i = 0; i < c->net_stride; ++i) {
            const int rc = launch_plain(c, from, bufs[i & 1], nullptr, s);
            if (rc) return rc;
            from = bufs[i & 1];
        }
        CK(launch_a_true_stride(D, from, Zt(0), AT, B, H, W, s));
    }

    // forward unroll: a_t, z_{t+1}, loss terms
    for (int t = 0; t < S; ++t) {
        CK(forward(Zt(t), A));
        if (t == 0) CK(launch_phys_term(D, P, A, AT, COEF, GA0, PART, B, H, W, s));
        CK(launch_train_euler(D, P, Zt(t), A, Zt(t + 1), B, H, W, s));
        CK(launch_data_term(D, P, Zt(t + 1), d_targets + (size_t)t * 3 * c->total_nodes, COEF + B, nullptr,
                            PART + (size_t)(t + 1) * blocks, B, H, W, s));
    }
    CK(launch_sum_partials(PART, (S + 1) * blocks, d_loss, s));
    if (!with_grad) return CLOTH_OK;

    // backward sweep, recomputing each step's activations (step checkpointing);
    // with segments, the states of a segment are recomputed from its
    // checkpoint when the sweep enters it (the same kernels: the same bits)
    CK(cudaMemsetAsync(GU, 0, sizeof(float) * 3 * NHW, s));
    CK(cudaMemsetAsync(GV, 0, sizeof(float) * 3 * NHW, s));
    int seg_loaded = -1;
    for (int t = S; t >= 1; --t) {
        if (k > 0 && (t - 1) / k != seg_loaded) {
            seg_loaded = (t - 1) / k;
            for (int q = seg_loaded * k; q < std::min(seg_loaded * k + k - 1, S); ++q) {
                CK(forward(Zt(q), A));
                CK(launch_train_euler(D, P, Zt(q), A, Zt(q + 1), B, H, W, s));
            }
        }
        CK(launch_data_term(D, P, Zt(t), d_targets + (size_t)(t - 1) * 3 * c->total_nodes, COEF + B, GU, nullptr,
                            B, H, W, s));
        CK(launch_euler_adjoint(D, P, GU, GV, t == 1 ? GA0 : nullptr, GA, GFP, B, H, W, s));
        CK(launch_pressure_vjp(D, Zt(t - 1), GFP, GE, GN, GU, B, H, W, s));
        CK(backward(Zt(t - 1), GA, GZ));
        CK(launch_add_gz(GZ, GU, GV, B, H, W, s));
    }
    return CLOTH_OK;
}

}  // namespace

extern "C" {

int cloth_train_loss(cloth_ctx* c, cloth_net* net, int32_t S, const float* d_targets, float alpha, float g_norm,
                     float* d_loss, float* d_grad_w, void* d_work, size_t bytes, void* stream)
{
    if (!c || !net) return CLOTH_EINVAL;
    if (net->precision != CLOTH_NET_FP32) return CLOTH_EUNSUPPORTED;
    if (S < 1) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const TrainWs L = train_ws(c, S);
    const int B = c->B, H = c->grids[0].rows, W = c->grids[0].cols;
    const int64_t NHW = (int64_t)B * H * W;
    float* SAVED = static_cast<float*>(d_work) + L.saved;
    auto forward = [&](const float* z, float* a) {   // a = cell(z_t), layer outputs into SAVED
        NetFwdArgs f{};
        f.src.z = z;
        f.w = net->d_w();
        f.t1 = SAVED + kSavT1 * NHW;
        f.t2 = SAVED + kSavT2 * NHW;
        f.s = SAVED + kSavS * NHW;
        f.a = a;
        f.N = B; f.H = H; f.W = W;
        f.status = c->d_status();
        return launch_net_forward_simt(f, s);
    };
    auto backward = [&](const float* z, const float* ga, float* gz) {
        cudaError_t e = forward(z, static_cast<float*>(d_work) + L.a);   // recompute the step's activations
        if (e != cudaSuccess) return e;
        return launch_net_backward_simt(net->d_w(), z, SAVED, ga, gz, net->d_part(), d_grad_w, B, H, W, c->d_status(),
                                        s);
    };
    return train_loss_impl(c, S, d_targets, alpha, g_norm, d_loss, d_work, bytes, s, forward, backward,
                           d_grad_w != nullptr);
}

int cloth_train_loss_pcell(cloth_ctx* c, const float* d_w, int32_t S, const float* d_targets, float alpha,
                           float g_norm, float* d_loss, float* d_grad_w, void* d_work, size_t bytes, void* stream)
{
    if (!c || !d_w || S < 1) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const TrainWs L = train_ws(c, S);
    const int B = c->B, H = c->grids[0].rows, W = c->grids[0].cols;
    float* PP = static_cast<float*>(d_work) + L.ppart;
    const ClothDesc* D = c->d_desc();
    auto forward = [&](const float* z, float* a) { return launch_pcell_fwd_z(D, d_w, z, a, B, H, W, s); };
    auto backward = [&](const float* z, const float* ga, float* gz) {
        return launch_pcell_bwd_z(D, d_w, z, ga, gz, PP, d_grad_w, B, H, W, s);
    };
    return train_loss_impl(c, S, d_targets, alpha, g_norm, d_loss, d_work, bytes, s, forward, backward,
                           d_grad_w != nullptr);
}

int net_adam_step(float* d_w, const float* d_grad, float* d_m, float* d_v, int32_t n, int32_t t, float lr,
                  float beta1, float beta2, float eps, void* stream)
{
    if (!d_w || !d_grad || !d_m || !d_v || n < 1 || t < 1) return CLOTH_EINVAL;
    CK(launch_adam(d_w, d_grad, d_m, d_v, nullptr, n, t, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

int net_adam_step_masked(float* d_w, const float* d_grad, float* d_m, float* d_v, const uint8_t* d_mask, int32_t n,
                         int32_t t, float lr, float beta1, float beta2, float eps, void* stream)
{
    if (!d_w || !d_grad || !d_m || !d_v || !d_mask || n < 1 || t < 1) return CLOTH_EINVAL;
    CK(launch_adam(d_w, d_grad, d_m, d_v, d_mask, n, t, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

namespace {
constexpr int kListsPcell = 2;   // lists_kind of the literal cell's tile list

std::vector<int4> pcell_tiles(const cloth_ctx* c)
{
    std::vector<int4> t;
    const int R = pcell_tile_rows(), Wt = pcell_tile_cols();
    for (int b = 0; b < c->B; ++b)
        for (int y0 = 0; y0 < c->grids[b].rows; y0 += R)
            for (int x0 = 0; x0 < c->grids[b].cols; x0 += Wt) t.push_back(make_int4(b, y0, x0, 0));
    return t;
}

int pcell_prepare(cloth_ctx* c, void* d_work, size_t bytes, cudaStream_t s, int* n_tiles)
{
    const std::vector<int4> tiles = pcell_tiles(c);
    if (bytes < sizeof(int4) * tiles.size()) return CLOTH_ENOMEM;
    if (reinterpret_cast<uintptr_t>(d_work) % kAlign) return CLOTH_EINVAL;
    if (c->lists_written != d_work || c->lists_kind != kListsPcell) {
        CK(cudaMemcpyAsync(d_work, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        c->lists_written = d_work;
        c->lists_kind = kListsPcell;
    }
    *n_tiles = (int)tiles.size();
    return CLOTH_OK;
}
}  // namespace

int cloth_pcell_workspace_size(const cloth_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return CLOTH_EINVAL;
    *bytes = align_up(sizeof(int4) * pcell_tiles(c).size(), kAlign);
    return CLOTH_OK;
}

int cloth_pcell_accel(cloth_ctx* c, const float* d_w, float* d_a, void* d_work, size_t bytes, void* stream)
{
    if (!c || !d_w || !d_a || !d_work) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int n = 0;
    const int rc = pcell_prepare(c, d_work, bytes, s, &n);
    if (rc) return rc;
    CK(launch_pcell(c->d_desc(), static_cast<const int4*>(d_work), n, d_w, c->d_state(c->cur), nullptr, d_a,
                    c->d_pins(), c->d_status(), s));
    return CLOTH_OK;
}

int cloth_step_pcell(cloth_ctx* c, const float* d_w, int32_t steps, void* d_work, size_t bytes, void* stream)
{
    if (!c || !d_w || !d_work || steps < 0) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int n = 0;
    const int rc = pcell_prepare(c, d_work, bytes, s, &n);
    if (rc) return rc;
    for (int st = 0; st < steps; ++st) {
        CK(launch_pcell(c->d_desc(), static_cast<const int4*>(d_work), n, d_w, c->d_state(c->cur),
                        c->d_state(c->cur ^ 1), nullptr, c->d_pins(), c->d_status(), s));
        c->cur ^= 1;
    }
    return CLOTH_OK;
}

int cloth_net_rollout_workspace_size(const cloth_ctx* c, int32_t precision, size_t* bytes)
{
    if (!c || !bytes) return CLOTH_EINVAL;
    size_t tiles = 0;
    int rc = cloth_net_workspace_size(c, precision, &tiles);
    if (rc) return rc;
    // + one scratch state buffer, two when a network step spans several
    // plain steps (the checked steps' plain reference ping-pongs)
    *bytes = align_up(tiles, kAlign) + (c->net_stride > 1 ? 2 : 1) * (c->L.state[1] - c->L.state[0]);
    return CLOTH_OK;
}

int cloth_rollout_net(cloth_ctx* c, const cloth_net* net, const cloth_net_rollout_opts* o, void* d_work, size_t bytes,
                      void* stream)
{
    if (!c || !net || !o || !d_work || o->steps < 0 || o->check_every < 0 || o->graph_chunk < 0) return CLOTH_EINVAL;
    if (o->check_every > 0 && !(o->residual_bound >= 0.f)) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t need = 0;
    int rc = cloth_net_rollout_workspace_size(c, net->precision, &need);
    if (rc) return rc;
    if (bytes < need) return CLOTH_ENOMEM;
    if (reinterpret_cast<uintptr_t>(d_work) % kAlign) return CLOTH_EINVAL;
    int n_tiles = 0;
    rc = net_tile_list(c, net, d_work, bytes, &n_tiles, s);
    if (rc) return rc;
    const int4* d_tiles = static_cast<const int4*>(d_work);
    float* scratch = reinterpret_cast<float*>(static_cast<char*>(d_work) + align_up(sizeof(int4) * n_tiles, kAlign));
    float* scratch2 = c->net_stride > 1 ? scratch + (c->L.state[1] - c->L.state[0]) / sizeof(float) : nullptr;
    const int k = c->net_stride;
    // k plain steps from src ending in dst, through `other` in between
    // (with `mode`, only the cloths in plain mode): step i writes dst when
    // k - i is even, `other` when it is odd
    auto plain_k = [&](const float* src, float* dst, float* other, const int32_t* mode, cudaStream_t ss) -> int {
        const float* from = src;
        for (int i = 1; i <= k; ++i) {
            float* to = (k - i) % 2 == 0 ? dst : other;
            const int r = launch_plain(c, from, to, mode, ss);
            if (r) return r;
            from = to;
        }
        return CLOTH_OK;
    };
    const int ce = o->check_every;
    auto one_step = [&](int st, cudaStream_t ss) -> int {
        const float* src = c->d_state(c->cur);
        float* dst = c->d_state(c->cur ^ 1);
        if (ce > 0 && st % ce == 0) {
            // both from the same state: the network step into the scratch
            // buffer, its k plain steps into dst, then keep, or latch to
            // plain, per cloth
            int r = launch_net_step(c, net, d_tiles, n_tiles, src, scratch, c->d_mode(), ss);
            if (r) return r;
            r = plain_k(src, dst, scratch2, nullptr, ss);
            if (r) return r;
            CK(launch_fallback_check(c->d_desc(), c->B, c->max_nodes, c->d_mode(), c->d_resid(), c->d_last(),
                                     o->residual_bound, scratch, dst, ss));
        } else {
            // cloths on the network: one network step; cloths on the plain
            // step: k plain steps (each kernel skips the other mode's cloths)
            int r = launch_net_step(c, net, d_tiles, n_tiles, src, dst, c->d_mode(), ss);
            if (r) return r;
            r = plain_k(src, dst, scratch, c->d_mode(), ss);
            if (r) return r;
        }
        c->cur ^= 1;
        return CLOTH_OK;
    };
    // graph chunks hold a whole number of check periods and an even number of
    // steps, so every replay starts on a check step with the same buffer
    int chunk = o->graph_chunk;
    if (chunk > 0) {
        const int period = ce > 0 ? (ce % 2 ? 2 * ce : ce) : 2;
        chunk = (chunk + period - 1) / period * period;
    }
    int done = 0;
    if (chunk > 0 && o->steps >= chunk) {
        // the graph is kept for later calls with the same network,
        // workspace, chunk, check period, bound and start buffer (the tile
        // list written above is the same for them)
        uint32_t bound_bits = 0;
        std::memcpy(&bound_bits, &o->residual_bound, sizeof(bound_bits));
        const cloth_ctx::NetGraphKey key{net, net->ws, net->precision, d_work, bytes, chunk, ce, bound_bits, c->cur};
        auto it = c->net_graphs.find(key);
        if (it == c->net_graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
            const int cur0 = c->cur;
            int r = CLOTH_OK;
            for (int i = 0; i < chunk && r == CLOTH_OK; ++i) r = one_step(i, c->cap);
            const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
            c->cur = cur0;
            if (r) { if (g) cudaGraphDestroy(g); return r; }
            if (e != cudaSuccess) return cuda_fail(e);
            const cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e2 != cudaSuccess) return cuda_fail(e2);
            it = c->net_graphs.emplace(key, ge).first;
        }
        while (o->steps - done >= chunk) {
            CK(cudaGraphLaunch(it->second, s));
            done += chunk;   // chunk is even: the current buffer is unchanged
        }
    }
    for (; done < o->steps; ++done) {
        const int r = one_step(done, s);
        if (r) return r;
    }
    return CLOTH_OK;
}

int cloth_modes(cloth_ctx* c, int32_t* d_mode, float* d_residual, void* stream)
{
    if (!c) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d_mode) CK(cudaMemcpyAsync(d_mode, c->d_mode(), sizeof(int32_t) * c->B, cudaMemcpyDeviceToDevice, s));
    if (d_residual) CK(cudaMemcpyAsync(d_residual, c->d_last(), sizeof(float) * c->B, cudaMemcpyDeviceToDevice, s));
    return CLOTH_OK;
}

int cloth_reset_modes(cloth_ctx* c, void* stream)
{
    if (!c) return CLOTH_EINVAL;
    CK(cudaMemsetAsync(c->ws + c->L.ctl, 0, 12 * (size_t)c->B, static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

int cloth_net_workspace_size(const cloth_ctx* c, int32_t precision, size_t* bytes)
{
    if (!c || !bytes || (precision != CLOTH_NET_FP32 && precision != CLOTH_NET_BF16)) return CLOTH_EINVAL;
    size_t n = 0;   // room for the list of any tile shape of the precision
    for (int v = 0; v < tile_choices(precision); ++v) n = std::max(n, shape_tiles(c, precision, v).size());
    *bytes = align_up(sizeof(int4) * n, kAlign);
    return CLOTH_OK;
}

int cloth_step_net(cloth_ctx* c, const cloth_net* net, int32_t steps, void* d_work, size_t bytes, void* stream)
{
    if (!c || !net || !d_work || steps < 0) return CLOTH_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_work) % kAlign) return CLOTH_EINVAL;
    return step_net_fused(c, net, steps, d_work, bytes, static_cast<cudaStream_t>(stream));
}

int cloth_workspace_size(int32_t B, const cloth_grid* grids, size_t* bytes)
{
    if (!bytes || !grids_ok(B, grids)) return CLOTH_EINVAL;
    *bytes = make_layout(B, grids).total;
    return CLOTH_OK;
}

int cloth_create(cloth_ctx** out, int32_t B, const cloth_grid* grids, const cloth_params* params,
                 const cloth_pins* pins, const cloth_sphere* spheres, float dt, void* d_workspace, size_t bytes,
                 void* stream)
{
    if (!out || !params || !d_workspace || !grids_ok(B, grids) || !(dt > 0.f) || !std::isfinite(dt))
        return CLOTH_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) return CLOTH_EINVAL;
    for (int b = 0; b < B; ++b)
        if (!(grids[b].spacing > 0.f) || !(grids[b].mass > 0.f)) return CLOTH_EINVAL;
    const Layout L = make_layout(B, grids);
    if (bytes < L.total) return CLOTH_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    cloth_ctx* c = new (std::nothrow) cloth_ctx;
    if (!c) return CLOTH_ENOMEM;
    c->B = B;
    c->ws = static_cast<char*>(d_workspace);
    c->L = L;
    c->grids.assign(grids, grids + B);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { delete c; return cuda_fail(e); }

    std::vector<uint32_t> pinmask(L.pin_words, 0u);
    std::vector<int2> pin_list;
    int64_t floats = 0, words = 0, nodes = 0;
    for (int b = 0; b < B; ++b) {
        const cloth_grid& g = grids[b];
        const cloth_params& p = params[b];
        ClothDesc d{};
        d.rows = g.rows;
        d.cols = g.cols;
        d.pitch = (int32_t)pitch_of(g.cols);
        d.pin_wpr = (d.pitch + 31) / 32;
        d.plane_off = floats;
        d.plane_stride = (int64_t)g.rows * d.pitch;
        d.pin_off = words;
        d.abi_off = nodes;
        d.h = g.spacing;
        d.m = g.mass;
        d.inv_m = 1.f / g.mass;
        d.dt = dt;
        d.dt_net = dt;
        d.k_struct = p.k_struct;
        d.k_shear = p.k_shear;
        d.k_bend = p.k_bend;
        d.mu = p.mu_spring;
        d.drag = p.drag;
        d.p_quarter = 0.25f * p.pressure;
        d.gx = p.gravity[0];
        d.gy = p.gravity[1];
        d.gz = p.gravity[2];
        if (p.mu_spring != 0.f) c->damp = true;
        d.sph_mu = -1.f;
        if (spheres && spheres[b].enabled) {
            if (!std::isfinite(spheres[b].friction)) { delete c; return CLOTH_EINVAL; }
            d.sph_mu = spheres[b].friction;
            d.sph_on = 1;
            d.sph_cx = spheres[b].center[0];
            d.sph_cy = spheres[b].center[1];
            d.sph_cz = spheres[b].center[2];
            d.sph_r = spheres[b].radius;
            d.sph_r2 = spheres[b].radius * spheres[b].radius;
        }
        int64_t pinned = 0;
        if (pins) {
            for (int a = 0; a < 3; ++a)
                if (!std::isfinite(pins[b].velocity[a])) { delete c; return CLOTH_EINVAL; }
            d.pin_vx = pins[b].velocity[0];
            d.pin_vy = pins[b].velocity[1];
            d.pin_vz = pins[b].velocity[2];
        }
        if (pins && pins[b].count > 0) {
            if (!pins[b].node) { delete c; return CLOTH_EINVAL; }
            for (int i = 0; i < pins[b].count; ++i) {
                const int32_t n = pins[b].node[i];
                if (n < 0 || (int64_t)n >= (int64_t)g.rows * g.cols) { delete c; return CLOTH_EINVAL; }
                const int r = n / g.cols, col = n % g.cols;
                uint32_t& wd = pinmask[words + (int64_t)r * d.pin_wpr + col / 32];
                if (!(wd & (1u << (col % 32)))) {
                    ++pinned;
                    pin_list.push_back(make_int2(b, n));
                }
                wd |= 1u << (col % 32);
            }
        }
        c->free_nodes.push_back((int64_t)g.rows * g.cols - pinned);
        c->desc.push_back(d);
        floats += align_up((size_t)(6 * d.plane_stride), kAlign / sizeof(float));
        words += (int64_t)g.rows * d.pin_wpr;
        nodes += (int64_t)g.rows * g.cols;
        c->max_nodes = std::max<int64_t>(c->max_nodes, (int64_t)g.rows * g.cols);
    }
    c->total_nodes = nodes;

    int rc = CLOTH_OK;
    e = cudaMemcpyAsync(c->d_desc(), c->desc.data(), sizeof(ClothDesc) * B, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && L.pin_words)
        e = cudaMemcpyAsync(c->d_pins(), pinmask.data(), sizeof(uint32_t) * L.pin_words, cudaMemcpyHostToDevice, s);
    c->n_pins = (int64_t)pin_list.size() <= L.pin_list_cap ? (int32_t)pin_list.size() : -1;
    if (e == cudaSuccess && c->n_pins > 0)
        e = cudaMemcpyAsync(c->d_pin_list(), pin_list.data(), sizeof(int2) * pin_list.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.state[0], 0, L.state[1] - L.state[0], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.state[1], 0, L.status - L.state[1], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.status, 0, L.total - L.status, s);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_fail(e);
    if (rc == CLOTH_OK) rc = set_work(c, pick_seg_rows(c), s);
    // the host copies above read pageable memory; wait so they are done
    // before the host vectors go out of scope
    if (rc == CLOTH_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_fail(e);
    if (rc != CLOTH_OK) {
        if (c->cap) cudaStreamDestroy(c->cap);
        delete c;
        return rc;
    }
    *out = c;
    return CLOTH_OK;
}

int cloth_set_state(cloth_ctx* c, const float* d_x, const float* d_v, void* stream)
{
    if (!c || !d_x) return CLOTH_EINVAL;
    CK(launch_set_state(c->d_desc(), c->B, c->max_nodes, nullptr, d_x, d_v, c->d_state(c->cur),
                        static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

int cloth_get_state(cloth_ctx* c, float* d_x, float* d_v, void* stream)
{
    if (!c) return CLOTH_EINVAL;
    if (!d_x && !d_v) return CLOTH_OK;
    CK(launch_get_state(c->d_desc(), c->B, c->max_nodes, nullptr, c->d_state(c->cur), d_x, d_v,
                        static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

int cloth_forces(cloth_ctx* c, float* d_f, void* stream)
{
    if (!c || !d_f) return CLOTH_EINVAL;
    return launch_step(c, true, d_f, static_cast<cudaStream_t>(stream));
}

int cloth_step_plain(cloth_ctx* c, int32_t steps, void* stream)
{
    if (!c || steps < 0) return CLOTH_EINVAL;
    for (int i = 0; i < steps; ++i) {
        const int rc = launch_step(c, false, nullptr, static_cast<cudaStream_t>(stream));
        if (rc) return rc;
    }
    return CLOTH_OK;
}

int cloth_rollout_plain(cloth_ctx* c, const cloth_rollout_opts* o, void* stream)
{
    if (!c || !o || o->steps < 0 || o->graph_chunk < 0) return CLOTH_EINVAL;
    if (o->d_record && o->record_every < 1) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o->d_record) {
        int frame = 0;
        for (int i = 1; i <= o->steps; ++i) {
            int rc = launch_step(c, false, nullptr, s);
            if (rc) return rc;
            if (i % o->record_every == 0) {
                rc = cloth_get_state(c, o->d_record + (int64_t)frame * 3 * c->total_nodes, nullptr, stream);
                if (rc) return rc;
                ++frame;
            }
        }
        return CLOTH_OK;
    }
    int chunk = o->graph_chunk;
    if (chunk & 1) ++chunk;
    int done = 0;
    if (chunk > 0 && o->steps >= chunk) {
        const auto key = std::make_pair(chunk, c->cur);
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
            const int cur0 = c->cur;
            int rc = CLOTH_OK;
            for (int i = 0; i < chunk && rc == CLOTH_OK; ++i) rc = launch_step(c, false, nullptr, c->cap);
            const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
            c->cur = cur0;   // capture only recorded the steps
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return cuda_fail(e);
            const cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e2 != cudaSuccess) return cuda_fail(e2);
            it = c->graphs.emplace(key, ge).first;
        }
        while (o->steps - done >= chunk) {
            CK(cudaGraphLaunch(it->second, s));
            done += chunk;   // chunk is even: the current buffer is unchanged
        }
    }
    for (; done < o->steps; ++done) {
        const int rc = launch_step(c, false, nullptr, s);
        if (rc) return rc;
    }
    return CLOTH_OK;
}

int cloth_set_launch(cloth_ctx* c, int32_t seg_rows, int32_t warps_per_sm, void* stream)
{
    if (!c || seg_rows < -1 || (seg_rows > 0 && seg_rows < kMinSegRows) || warps_per_sm < -1 || warps_per_sm > 64)
        return CLOTH_EINVAL;
    if (warps_per_sm != 0) c->warps_per_sm = warps_per_sm > 0 ? warps_per_sm : 0;
    drop_graphs(c);
    const int seg = seg_rows > 0 ? seg_rows : (seg_rows < 0 ? 0 : c->seg_rows);
    const int rc = set_work(c, seg, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

int cloth_tune_launch(cloth_ctx* c, int32_t n, const int32_t* seg_rows, const int32_t* warps_per_sm, int32_t warmup,
                      int32_t steps, float* us_out, int32_t* best, void* stream)
{
    if (!c || n < 1 || !seg_rows || !warps_per_sm || !us_out || !best || warmup < 0 || steps < 1) return CLOTH_EINVAL;
    for (int i = 0; i < n; ++i) {
        const int R = seg_rows[i], w = warps_per_sm[i];
        if (!(R == -1 || R >= kMinSegRows) || !(w == -1 || (w >= 1 && w <= 64))) return CLOTH_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    drop_graphs(c);
    // apply candidate i as cloth_set_launch would (-1: balanced / default)
    auto apply = [&](int i) {
        c->warps_per_sm = warps_per_sm[i] > 0 ? warps_per_sm[i] : 0;
        return set_work(c, seg_rows[i] > 0 ? seg_rows[i] : 0, s);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CLOTH_OK;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    // every timed step reads the current state and writes the other buffer,
    // so the state the caller sees does not move
    const float* src = c->d_state(c->cur);
    float* dst = c->d_state(c->cur ^ 1);
    // each candidate's `steps` steps are timed as one CUDA graph, as rollouts
    // replay them (eager launches rank the shapes differently)
    for (int i = 0; i < n && rc == CLOTH_OK && ce == cudaSuccess; ++i) {
        rc = apply(i);
        if (rc) break;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        if ((ce = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        for (int k = 0; k < steps && rc == CLOTH_OK; ++k) rc = launch_plain(c, src, dst, nullptr, c->cap);
        const cudaError_t ec = cudaStreamEndCapture(c->cap, &g);
        if (rc == CLOTH_OK && (ce = ec) == cudaSuccess) ce = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        for (int k = 0; k <= warmup && rc == CLOTH_OK && ce == cudaSuccess; ++k)   // at least one untimed replay
            ce = cudaGraphLaunch(ge, s);
        constexpr int kReplays = 2;   // timed
        if (rc == CLOTH_OK && ce == cudaSuccess) ce = cudaEventRecord(e0, s);
        for (int k = 0; k < kReplays && rc == CLOTH_OK && ce == cudaSuccess; ++k) ce = cudaGraphLaunch(ge, s);
        if (rc == CLOTH_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, s);
        if (rc == CLOTH_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (rc == CLOTH_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ge) cudaGraphExecDestroy(ge);
        if (rc || ce != cudaSuccess) break;
        us_out[i] = ms * 1000.f / (float)(kReplays * steps);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ce != cudaSuccess) return cuda_fail(ce);
    if (rc) return rc;
    int b = 0;
    for (int i = 1; i < n; ++i)
        if (us_out[i] < us_out[b]) b = i;
    *best = b;
    rc = apply(b);
    if (rc) return rc;
    CK(cudaStreamSynchronize(s));
    return CLOTH_OK;
}

int cloth_net_tile_choices(int32_t precision, int32_t* rows, int32_t* cols, int32_t* kinds, int32_t capacity,
                           int32_t* count)
{
    if (!count || capacity < 0 || (capacity > 0 && (!rows || !cols || !kinds))) return CLOTH_EINVAL;
    if (precision != CLOTH_NET_FP32 && precision != CLOTH_NET_BF16) return CLOTH_EINVAL;
    *count = tile_choices(precision);
    for (int v = 0; v < *count && v < capacity; ++v) tile_shape(precision, v, &rows[v], &cols[v], &kinds[v]);
    return CLOTH_OK;
}

int cloth_set_net_tile(cloth_ctx* c, int32_t precision, int32_t choice)
{
    if (!c || (precision != CLOTH_NET_FP32 && precision != CLOTH_NET_BF16)) return CLOTH_EINVAL;
    if (choice < 0 || choice >= tile_choices(precision)) return CLOTH_EINVAL;
    if (choice != tile_variant(c, precision)) {
        drop_graphs(c);   // the captured network steps use the old shape
        tile_variant(c, precision) = choice;
    }
    return CLOTH_OK;
}

int cloth_get_net_tile(const cloth_ctx* c, int32_t precision, int32_t* choice)
{
    if (!c || !choice || (precision != CLOTH_NET_FP32 && precision != CLOTH_NET_BF16)) return CLOTH_EINVAL;
    *choice = tile_variant(c, precision);
    return CLOTH_OK;
}

int cloth_tune_net(cloth_ctx* c, const cloth_net* net, int32_t warmup, int32_t steps, float* us_out,
                   int32_t* best, void* d_work, size_t bytes, void* stream)
{
    if (!c || !net || !us_out || !best || !d_work || warmup < 0 || steps < 1) return CLOTH_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_work) % kAlign) return CLOTH_EINVAL;
    size_t need = 0;
    int rc = cloth_net_workspace_size(c, net->precision, &need);
    if (rc) return rc;
    if (bytes < need) return CLOTH_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    drop_graphs(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    // every timed step reads the current state and writes the other buffer,
    // so the state the caller sees does not move
    const float* src = c->d_state(c->cur);
    float* dst = c->d_state(c->cur ^ 1);
    const int nv = tile_choices(net->precision);
    int& var = tile_variant(c, net->precision);
    for (int v = 0; v < nv && rc == CLOTH_OK && ce == cudaSuccess; ++v) {
        var = v;
        int n_tiles = 0;
        rc = net_tile_list(c, net, d_work, bytes, &n_tiles, s);
        const int4* tl = static_cast<const int4*>(d_work);
        for (int k = 0; k < warmup && rc == CLOTH_OK; ++k) rc = launch_net_step(c, net, tl, n_tiles, src, dst, nullptr, s);
        if (rc) break;
        if ((ce = cudaEventRecord(e0, s)) != cudaSuccess) break;
        for (int k = 0; k < steps && rc == CLOTH_OK; ++k) rc = launch_net_step(c, net, tl, n_tiles, src, dst, nullptr, s);
        if (rc) break;
        if ((ce = cudaEventRecord(e1, s)) != cudaSuccess) break;
        if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        if ((ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        us_out[v] = ms * 1000.f / (float)steps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ce != cudaSuccess) { var = 0; return cuda_fail(ce); }
    if (rc) { var = 0; return rc; }
    int b = 0;
    for (int v = 1; v < nv; ++v)
        if (us_out[v] < us_out[b]) b = v;
    var = b;
    *best = b;
    return CLOTH_OK;
}

int cloth_set_boundary(cloth_ctx* c, int32_t b, const float* pin_velocity, float sphere_friction, void* stream)
{
    if (!c || b < 0 || b >= c->B || !pin_velocity || !std::isfinite(sphere_friction)) return CLOTH_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(pin_velocity[a])) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ClothDesc& d = c->desc[b];
    d.pin_vx = pin_velocity[0];
    d.pin_vy = pin_velocity[1];
    d.pin_vz = pin_velocity[2];
    d.sph_mu = sphere_friction;
    CK(cudaMemcpyAsync(c->d_desc() + b, &d, sizeof(ClothDesc), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return CLOTH_OK;
}

namespace {
struct ImplWs {
    size_t vecs, fabi, part, scal, blk, total;
};
ImplWs impl_ws(const cloth_ctx* c)
{
    ImplWs w{};
    size_t off = 0;
    auto take = [&](size_t floats) { const size_t o = off; off = align_up(off + floats, kAlign / sizeof(float)); return o; };
    w.vecs = take((size_t)4 * c->L.state_floats);
    w.fabi = take((size_t)3 * c->total_nodes);
    w.part = take((size_t)c->B * implicit_grid_x(c->max_nodes));
    w.scal = take((size_t)3 * c->B);
    w.blk = take((size_t)c->B + 1);   // int32 block starts
    w.total = off * sizeof(float);
    return w;
}
}  // namespace

int cloth_implicit_workspace_size(const cloth_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return CLOTH_EINVAL;
    *bytes = impl_ws(c).total;
    return CLOTH_OK;
}

int cloth_step_implicit(cloth_ctx* c, int32_t steps, int32_t stride, int32_t cg_iters, void* d_work, size_t bytes,
                        void* stream)
{
    if (!c || steps < 0 || stride < 1 || stride > kMaxNetStride || cg_iters < 0 || cg_iters > 100000 || !d_work)
        return CLOTH_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_work) % kAlign) return CLOTH_EINVAL;
    const ImplWs w = impl_ws(c);
    if (bytes < w.total) return CLOTH_ENOMEM;
    for (const ClothDesc& d : c->desc)   // the kernels index a cloth's 6 planes in 32 bits
        if (6 * d.plane_stride >= ((int64_t)1 << 31)) return CLOTH_EUNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* ws = static_cast<float*>(d_work);
    const float h = (float)stride * c->desc[0].dt;
    if (c->impl_blk.empty()) {   // the flat grid's first block of each cloth
        const int64_t tb = implicit_block_nodes();
        c->impl_blk.push_back(0);
        for (int b = 0; b < c->B; ++b)
            c->impl_blk.push_back(c->impl_blk.back() +
                                  (int32_t)(((int64_t)c->grids[b].rows * c->grids[b].cols + tb - 1) / tb));
    }
    int32_t* blk = reinterpret_cast<int32_t*>(ws + w.blk);
    CK(cudaMemcpyAsync(blk, c->impl_blk.data(), sizeof(int32_t) * (c->B + 1), cudaMemcpyHostToDevice, s));
    for (int i = 0; i < steps; ++i) {
        const int rc = launch_step(c, true, ws + w.fabi, s);   // explicit forces at the current state
        if (rc) return rc;
        CK(launch_implicit_step(c->d_desc(), c->d_pins(), c->B, c->max_nodes, blk, c->impl_blk.back(),
                                c->d_state(c->cur), ws + w.fabi,
                                c->d_state(c->cur ^ 1), ws + w.vecs, c->L.state_floats, ws + w.part, ws + w.scal, h,
                                cg_iters, c->d_status(), s));
        c->cur ^= 1;
    }
    return CLOTH_OK;
}

int cloth_set_train_segment(cloth_ctx* c, int32_t k)
{
    if (!c || k < 0) return CLOTH_EINVAL;
    c->train_seg = k;
    return CLOTH_OK;
}

int cloth_set_net_stride(cloth_ctx* c, int32_t k, void* stream)
{
    if (!c || k < 1 || k > kMaxNetStride) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (auto& d : c->desc) d.dt_net = (float)k * d.dt;
    if (k != c->net_stride) drop_graphs(c);   // a network step's plain steps are captured
    c->net_stride = k;
    CK(cudaMemcpyAsync(c->d_desc(), c->desc.data(), sizeof(ClothDesc) * c->B, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return CLOTH_OK;
}

int cloth_get_launch(const cloth_ctx* c, int32_t* seg_rows, int32_t* warps_per_sm, int32_t* n_units)
{
    if (!c) return CLOTH_EINVAL;
    if (seg_rows) *seg_rows = c->seg_rows;
    if (warps_per_sm) *warps_per_sm = c->warps_per_sm;
    if (n_units) *n_units = c->n_units;
    return CLOTH_OK;
}

int cloth_topology(cloth_ctx* c, int32_t b, uint16_t* d_mask, void* stream)
{
    if (!c || !d_mask || b < 0 || b >= c->B) return CLOTH_EINVAL;
    CK(launch_topology(c->d_desc(), b, c->grids[b].rows, c->grids[b].cols, d_mask, static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

int cloth_selftest_wait_timeout(cloth_ctx* c, int32_t polls, void* stream)
{
    if (!c || polls < 1) return CLOTH_EINVAL;
    CK(launch_wait_timeout_selftest(c->d_status(), (uint32_t)polls, static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

int cloth_status(cloth_ctx* c, int32_t* h_status, int32_t clear, void* stream)
{
    if (!c || !h_status) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(h_status, c->d_status(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (clear) {
        CK(cudaMemsetAsync(c->d_status(), 0, sizeof(int32_t), s));
        CK(cudaStreamSynchronize(s));
    }
    return CLOTH_OK;
}

int cloth_info(const cloth_ctx* c, int32_t* B, int64_t* total_nodes)
{
    if (!c) return CLOTH_EINVAL;
    if (B) *B = c->B;
    if (total_nodes) *total_nodes = c->total_nodes;
    return CLOTH_OK;
}

void cloth_destroy(cloth_ctx* c)
{
    if (!c) return;
    drop_graphs(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

const char* cloth_strerror(int code)
{
    switch (code) {
    case CLOTH_OK: return "ok";
    case CLOTH_EINVAL: return "invalid argument";
    case CLOTH_ENOMEM: return "workspace too small";
    case CLOTH_ECUDA: return "CUDA runtime error";
    case CLOTH_ENONFINITE: return "non-finite state";
    case CLOTH_ETIMEOUT: return "device wait timed out";
    case CLOTH_EUNSUPPORTED: return "unsupported request";
    default: return "unknown error";
    }
}

int cloth_last_cuda_error(void)
{
    const int n = cloth::net_last_cuda_error();
    return g_last_cuda ? g_last_cuda : n;
}

}  // extern "C"
