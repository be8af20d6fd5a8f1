// net_forward_static: the FP32 cell forward without any device allocation.
//
// The ordinary net_forward keeps the two 64-channel layer outputs of the
// trunk (phi1, xi1 and phi, xi) in a buffer the caller allocates.  Some
// callers cannot allocate device memory on demand: plug-ins that run inside
// a host application which reserves the whole GPU memory budget up front
// and forbids allocations afterwards, and real-time frame loops in which a
// cudaMalloc could stall a frame.  For them this entry point keeps those
// layer outputs in one file-scope device array of fixed size instead.  Its
// limits: at most kStaticMaxNodes nodes (N * H * W) per call; every GPU
// that loads the library holds the array (8 MiB) until the process exits;
// every call on a device shares the same array, so calls whose work
// overlaps on that GPU (different streams, or host threads) race with each
// other.
#include <mutex>

#include "../../include/cloth.h"
#include "net_internal.cuh"

using namespace cloth;

namespace {

constexpr int64_t kStaticMaxNodes = CLOTH_NET_STATIC_MAX_NODES;
constexpr int64_t kStaticFloatsPerNode = 128;   // phi1, xi1 (64) + phi, xi (64)

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; kernels receive the device address cudaGetSymbolAddress reports.
__device__ __align__(256) float g_net_static_scratch[kStaticMaxNodes * kStaticFloatsPerNode];

struct DeviceScratch {
    bool ready = false;
    float* ptr = nullptr;
};

std::mutex g_mu;
DeviceScratch g_dev[64];

// CUDA failures go where cloth_last_cuda_error reads them.
int static_cuda_fail(cudaError_t e)
{
    net_record_cuda_error((int)e);
    return CLOTH_ECUDA;
}

// Device address of the scratch on the current device, looked up (and the
// kernels' shared-memory limits raised) the first time a device is used.
// Both are kept for the life of the process: a cudaDeviceReset after that
// first call would leave them stale, so it is not supported.
int scratch_address(float** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_cuda_fail(e);
    if (dev < 0 || dev >= 64) return CLOTH_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev[dev].ready) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_net_static_scratch);
        if (e == cudaSuccess) e = net_simt_init();
        if (e != cudaSuccess) return static_cuda_fail(e);
        g_dev[dev].ptr = static_cast<float*>(p);
        g_dev[dev].ready = true;
    }
    *out = g_dev[dev].ptr;
    return CLOTH_OK;
}

}  // namespace

extern "C" int net_forward_static(const float* d_blob, const float* d_z, float* d_a, int32_t N, int32_t H,
                                  int32_t W, void* stream)
{
    if (!d_blob || !d_z || !d_a || N < 1 || H < 1 || W < 1 || N > 32767) return CLOTH_EINVAL;
    const int64_t nodes = (int64_t)N * H * W;
    if (nodes > kStaticMaxNodes) return CLOTH_EINVAL;
    float* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != CLOTH_OK) return rc;
    // every scratch element the kernels read is written earlier in the same
    // call, so nothing has to be cleared between calls
    NetFwdArgs f{};
    f.src.z = d_z;
    f.w = d_blob;
    f.t1 = scratch;
    f.t2 = scratch + 64 * nodes;
    f.s = nullptr;
    f.a = d_a;
    f.N = N;
    f.H = H;
    f.W = W;
    const cudaError_t e = launch_net_forward_simt(f, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return static_cuda_fail(e);
    return CLOTH_OK;
}
