// Launchers of the training kernels (train.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cloth_internal.cuh"

namespace cloth {

int train_blocks(int H, int W, int B);
cudaError_t launch_state_to_z(const ClothDesc* d, const float* state, float* z, int B, int H, int W, cudaStream_t s);
cudaError_t launch_a_true_stride(const ClothDesc* d, const float* state_k, const float* z, float* at, int B, int H,
                                 int W, cudaStream_t s);
cudaError_t launch_a_true(const ClothDesc* d, const float* f_abi, const float* z, float* at, int B, int H, int W,
                          cudaStream_t s);
cudaError_t launch_train_euler(const ClothDesc* d, const uint32_t* pins, const float* z, const float* a, float* zn,
                               int B, int H, int W, cudaStream_t s);
cudaError_t launch_data_term(const ClothDesc* d, const uint32_t* pins, const float* z, const float* xt,
                             const float* coef, float* gu, float* part, int B, int H, int W, cudaStream_t s);
cudaError_t launch_phys_term(const ClothDesc* d, const uint32_t* pins, const float* a0, const float* at,
                             const float* coef, float* ga0, float* part, int B, int H, int W, cudaStream_t s);
cudaError_t launch_sum_partials(const float* part, int count, float* out, cudaStream_t s);
cudaError_t launch_euler_adjoint(const ClothDesc* d, const uint32_t* pins, const float* gu, float* gv,
                                 const float* ga0, float* ga, float* gfp, int B, int H, int W, cudaStream_t s);
cudaError_t launch_pressure_vjp(const ClothDesc* d, const float* z, const float* gfp, float* ge, float* gn, float* gu,
                                int B, int H, int W, cudaStream_t s);
cudaError_t launch_add_gz(const float* gz, float* gu, float* gv, int B, int H, int W, cudaStream_t s);
cudaError_t launch_adam(float* w, const float* g, float* m, float* v, const uint8_t* mask, int n, int t, float lr,
                        float b1, float b2, float eps, cudaStream_t s);
// The literal cell on the training layout (pcell_train.cu).
int pcell_train_blocks(int H, int W, int B);
cudaError_t launch_pcell_fwd_z(const ClothDesc* d, const float* w, const float* z, float* a, int B, int H, int W,
                               cudaStream_t s);
cudaError_t launch_pcell_bwd_z(const ClothDesc* d, const float* w, const float* z, const float* ga, float* gz,
                               float* part, float* grad_w, int B, int H, int W, cudaStream_t s);

}  // namespace cloth
