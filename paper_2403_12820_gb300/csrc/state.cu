// State conversion between the packed ABI layout (per cloth [rows][cols][3]
// floats, cloths back to back) and the internal SoA planes of the
// displacement u = x - X and velocity v; and the topology probe.
//
// The rest position X = (c h, r h, 0) is formed in FP64 (exact: c and h are
// both representable), so u = fl32(x - X) and x = fl32(X + u) add no error
// beyond the final rounding.
#include "cloth_internal.cuh"

namespace cloth {
namespace {

__global__ void set_state_kernel(const ClothDesc* __restrict__ desc, const float* __restrict__ x,
                                 const float* __restrict__ v, float* __restrict__ state)
{
    const ClothDesc& D = desc[blockIdx.y];
    const int64_t n = (int64_t)D.rows * D.cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / D.cols), c = (int)(i % D.cols);
        const int64_t src = (D.abi_off + i) * 3;
        const int64_t dst = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
        const double X = (double)c * (double)D.h, Y = (double)r * (double)D.h;
        state[dst] = (float)((double)x[src + 0] - X);
        state[dst + D.plane_stride] = (float)((double)x[src + 1] - Y);
        state[dst + 2 * D.plane_stride] = x[src + 2];
        for (int k = 0; k < 3; ++k) state[dst + (3 + k) * D.plane_stride] = v ? v[src + k] : 0.f;
    }
}

__global__ void get_state_kernel(const ClothDesc* __restrict__ desc, const float* __restrict__ state,
                                 float* __restrict__ x, float* __restrict__ v)
{
    const ClothDesc& D = desc[blockIdx.y];
    const int64_t n = (int64_t)D.rows * D.cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / D.cols), c = (int)(i % D.cols);
        const int64_t dst = (D.abi_off + i) * 3;
        const int64_t src = D.plane_off + (int64_t)r * D.pitch + col_pos(c);
        if (x) {
            x[dst + 0] = (float)((double)c * (double)D.h + (double)state[src]);
            x[dst + 1] = (float)((double)r * (double)D.h + (double)state[src + D.plane_stride]);
            x[dst + 2] = state[src + 2 * D.plane_stride];
        }
        if (v)
            for (int k = 0; k < 3; ++k) v[dst + k] = state[src + (3 + k) * D.plane_stride];
    }
}

// Spring s exists iff both ends are inside the grid; offsets (dr, dc) in the
// order E, N, W, S, NE, NW, SW, SE, 2E, 2N, 2W, 2S.
__constant__ int8_t kOff[12][2] = {{0, 1}, {1, 0}, {0, -1}, {-1, 0}, {1, 1}, {1, -1},
                                   {-1, -1}, {-1, 1}, {0, 2}, {2, 0}, {0, -2}, {-2, 0}};

__global__ void topology_kernel(int rows, int cols, uint16_t* __restrict__ mask)
{
    const int64_t n = (int64_t)rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        unsigned m = 0;
        for (int s = 0; s < 12; ++s) {
            const int r2 = r + kOff[s][0], c2 = c + kOff[s][1];
            if ((unsigned)r2 < (unsigned)rows && (unsigned)c2 < (unsigned)cols) m |= 1u << s;
        }
        mask[i] = (uint16_t)m;
    }
}

int grid_for(int64_t n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

cudaError_t launch_set_state(const ClothDesc* desc, int32_t B, int64_t max_nodes, const int64_t*, const float* x,
                             const float* v, float* state, cudaStream_t s)
{
    dim3 grid(grid_for(max_nodes), B);
    set_state_kernel<<<grid, 256, 0, s>>>(desc, x, v, state);
    return cudaGetLastError();
}

cudaError_t launch_get_state(const ClothDesc* desc, int32_t B, int64_t max_nodes, const int64_t*, const float* state,
                             float* x, float* v, cudaStream_t s)
{
    dim3 grid(grid_for(max_nodes), B);
    get_state_kernel<<<grid, 256, 0, s>>>(desc, state, x, v);
    return cudaGetLastError();
}

cudaError_t launch_topology(const ClothDesc*, int32_t, int32_t rows, int32_t cols, uint16_t* mask, cudaStream_t s)
{
    topology_kernel<<<grid_for((int64_t)rows * cols), 256, 0, s>>>(rows, cols, mask);
    return cudaGetLastError();
}

}  // namespace cloth
