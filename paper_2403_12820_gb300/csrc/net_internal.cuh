// Internal structures of the CNN cell (Sec. 3.2, Eq. 6-7) in libcloth.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cloth_internal.cuh"

namespace cloth {

// Weight blob offsets (floats): W1[32][6][3][3], W2[32][32][3][3],
// WL[3][32][3][3], bL[3], P[32][32], WN[3][32], WD[3][32], in_scale[6],
// out_scale[3].
constexpr int kC = 32;
constexpr int kOffW1 = 0;
constexpr int kOffW2 = kOffW1 + kC * 6 * 9;
constexpr int kOffWL = kOffW2 + kC * kC * 9;
constexpr int kOffBL = kOffWL + 3 * kC * 9;
constexpr int kOffP = kOffBL + 3;
constexpr int kOffWN = kOffP + kC * kC;
constexpr int kOffWD = kOffWN + 3 * kC;
constexpr int kParams = kOffWD + 3 * kC;   // 13027 trainable
constexpr int kOffIns = kParams;
constexpr int kOffOuts = kOffIns + 6;
constexpr int kBlob = kOffOuts + 3;        // 13036

// Blocks of the weight-gradient kernels; each writes one partial row of
// kParams floats that a fixed-order reduction sums.
constexpr int kWgradBlocks = 512;

// Saved activations of net_forward for net_backward, per node (floats), as
// NCHW regions of the N images:
//   T1 [N][2][32] (phi1, xi1)   T2 [N][2][32] (phi, xi)   S [N][32] (s)
//   G2 [N][2][32] (d phi, d xi) GT [N][32] (d t)          GY [N][3] (d y)
// net_backward writes d phi1, d xi1 over T2 once T2 is no longer needed.
constexpr int64_t kSavT1 = 0, kSavT2 = 64, kSavS = 128, kSavG2 = 160, kSavGT = 224, kSavGY = 256;
constexpr int64_t kSavedPerNode = 260;

// Where the cell reads its 6 input channels from: NCHW z [N][6][H][W].
struct NetSrc {
    const float* z;
};

struct NetFwdArgs {
    NetSrc src;
    const float* w;     // FP32 weight blob (device)
    float* t1;          // [N][2][32][H][W]
    float* t2;          // [N][2][32][H][W]
    float* s;           // [N][32][H][W] or nullptr
    float* a;           // [N][3][H][W]
    int N, H, W;
    int32_t* status;    // status word for a timed-out tensor-core wait; null: the second
                        // convolution runs on the CUDA cores
};

cudaError_t launch_net_forward_simt(const NetFwdArgs& f, cudaStream_t s);
cudaError_t launch_net_backward_simt(const float* w, const float* z, float* saved, const float* ga, float* gz,
                                     float* partials, float* gw, int N, int H, int W, int32_t* status, cudaStream_t s);
// The 32 -> 32 3x3 convolution W2 (*) (or its adjoint, `transposed`) on the
// tensor cores at FP32 precision (conv_tc.cu): NCHW images of 32 channels.
cudaError_t conv32_tc_init();
cudaError_t launch_conv32_tc(const float* in, float* out, const float* w, bool transposed, int images, int H, int W,
                             int32_t* status, cudaStream_t s);
cudaError_t net_simt_init();
int net_last_cuda_error();
// Record a CUDA failure of a network entry point for cloth_last_cuda_error.
void net_record_cuda_error(int e);
// One column of the trunk's composite kernels (Eq. 6 folded into Eq. 7):
// G_n W2_a W1_b[:, i] for 3x3 taps a (W2) and b (W1) and input channel i,
// where G_n is P's row n (n < 32), WL's tap tl and output co
// (n = 32 + 3 tl + co < 59) or, for n >= 64, the identity on channel n - 64
// (the velocity features xi).  Summed over a + b = c it is the 5x5
// composite tap c; single (a, b) pairs give the edge and corner terms.
__device__ inline float trunk_composite(const float* __restrict__ w, int n, int i, int a, int b)
{
    float s = 0.f;
    if (n >= 64) {
        const int k = n - 64;
        for (int j = 0; j < kC; ++j) s = fmaf(w[kOffW2 + (k * kC + j) * 9 + a], w[kOffW1 + (j * 6 + i) * 9 + b], s);
        return s;
    }
    for (int k = 0; k < kC; ++k) {
        const float gk = n < 32 ? w[kOffP + n * kC + k] : w[kOffWL + ((n - 32) % 3 * kC + k) * 9 + (n - 32) / 3];
        float d = 0.f;
        for (int j = 0; j < kC; ++j) d = fmaf(w[kOffW2 + (k * kC + j) * 9 + a], w[kOffW1 + (j * 6 + i) * 9 + b], d);
        s = fmaf(gk, d, s);
    }
    return s;
}

// tanh from the identity tanh(x) = 1 - 2 / (e^(2x) + 1), with the hardware
// base-2 exponential (e^(2x) = 2^(2x log2 e)) and reciprocal: an absolute
// error of about 1e-6 (both approximations are within a few units of the
// last place), against the FP32 step's 1e-4 tolerance on the acceleration.
// Large |x| saturate cleanly: e^(2x) = inf gives 1, e^(2x) = 0 gives -1.
__device__ __forceinline__ float tanh_exp(float x)
{
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(x * 2.8853900817779268f));   // 2 log2(e)
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.f));
    return fmaf(-2.f, r, 1.f);
}

// Tensor-core (tcgen05, BF16) fused cell / network step (net_tc.cu): tiles
// of net_tc_variant_rows(v) x net_tc_tile_cols() output nodes for one of
// net_tc_variants() BF16 tile shapes v (0: the default), and the FP32 step
// as three BF16 products per term (hi hi + hi lo + lo hi, "split") on tiles
// of net_tc_split_rows(k) rows for one of net_tc_split_variants() shapes k;
// launch_net_tc_step takes v, or k when `split`.
cudaError_t net_tc_init();
int net_tc_pack_bytes();
int net_tc_edge_offset();   // bytes from the pack's start to the FP32 edge and corner terms
int net_tc_tile_cols();
int net_tc_variants();
int net_tc_variant_rows(int v);
int net_tc_split_variants();
int net_tc_split_rows(int k);
cudaError_t launch_pack_bf16(const float* w, void* wpack, cudaStream_t s);
cudaError_t launch_net_tc_step(int variant, bool split, const void* wpack, const float* w, const ClothDesc* desc,
                               const int4* tiles, int n_tiles, const float* src, float* dst, const uint32_t* pinmask,
                               int32_t* status, int grid, cudaStream_t s, const int32_t* mode = nullptr);
cudaError_t launch_net_tc_forward(const void* wpack, const float* w, const float* z, float* out, int N, int H, int W,
                                  int32_t* status, int grid, cudaStream_t s);
// FP32 fused network step with the composite trunk (net_comp.cu): tiles of
// net_comp_tile_rows() x net_comp_variant_cols(v) output nodes for one of
// net_comp_variants() tile shapes v (0: the default; the launch tuner picks
// among them), net_comp_blocks_per_sm(v) resident blocks per SM; its
// composite weights (net_comp_pack_floats() floats) follow the tensor-core
// operands in the pack, and it reads their FP32 edge and corner terms.
int net_comp_tile_rows();
int net_comp_variants();
int net_comp_variant_cols(int v);
int net_comp_blocks_per_sm(int v);
int net_comp_pack_floats();
cudaError_t net_comp_init();
cudaError_t launch_pack_comp(const float* w, float* out, cudaStream_t s);
cudaError_t launch_net_comp_step(int variant, const float* w, const float* wf, const float* ke, const ClothDesc* desc,
                                 const int4* tiles, int n_tiles, const float* src, float* dst,
                                 const uint32_t* pinmask, int32_t* status, int grid, cudaStream_t s,
                                 const int32_t* mode = nullptr);


// Host side of a network handle (include/cloth.h: cloth_net).
struct NetLayout {
    size_t blob, part, pack, status, total;
};
inline NetLayout net_layout()
{
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    NetLayout L{};
    size_t off = 0;
    L.blob = off; off = al(off + sizeof(float) * kBlob);
    L.part = off; off = al(off + sizeof(float) * (size_t)kWgradBlocks * kParams);
    // packed tensor-core operands, then the FP32 composite weights (d_comp)
    L.pack = off; off = al(off + al((size_t)net_tc_pack_bytes()) + sizeof(float) * (size_t)net_comp_pack_floats());
    L.status = off; off = al(off + 64);
    L.total = off;
    return L;
}

}  // namespace cloth

struct cloth_net {
    int32_t precision = 0;
    char* ws = nullptr;
    cloth::NetLayout L{};
    float* d_w() const { return reinterpret_cast<float*>(ws + L.blob); }
    float* d_part() const { return reinterpret_cast<float*>(ws + L.part); }
    void* d_pack() const { return ws + L.pack; }
    // the FP32 composite weights after the tensor-core operands, and the
    // FP32 edge and corner terms inside them
    float* d_comp() const { return reinterpret_cast<float*>(ws + L.pack + (cloth::net_tc_pack_bytes() + 255) / 256 * 256); }
    // (net_layout reserves exactly these two parts, in this order)
    const float* d_edge() const { return reinterpret_cast<const float*>(ws + L.pack + cloth::net_tc_edge_offset()); }
    int32_t* d_status() const { return reinterpret_cast<int32_t*>(ws + L.status); }
    int sm_count = 0;
};
