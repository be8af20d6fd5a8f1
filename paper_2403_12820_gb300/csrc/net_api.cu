// Host implementation of the CNN-cell entry points of include/cloth.h.
#include <cmath>
#include <mutex>
#include <new>

#include "../../include/cloth.h"
#include "net_internal.cuh"

using namespace cloth;

namespace {

thread_local int g_net_cuda = 0;

int net_cuda_fail(cudaError_t e)
{
    g_net_cuda = (int)e;
    return CLOTH_ECUDA;
}

#define NCK(expr)                                        \
    do {                                                 \
        cudaError_t e__ = (expr);                        \
        if (e__ != cudaSuccess) return net_cuda_fail(e__); \
    } while (0)

// Kernel attributes are per device; set them once for every device used.
int ensure_init()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    NCK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return CLOTH_EUNSUPPORTED;
    if (!done[dev]) {
        NCK(net_simt_init());
        NCK(net_tc_init());
        NCK(net_comp_init());
        done[dev] = true;
    }
    return CLOTH_OK;
}

bool dims_ok(int32_t N, int32_t H, int32_t W)
{
    return N >= 1 && H >= 1 && W >= 1 && N <= 32767 && H <= (1 << 16) && W <= (1 << 16);
}

}  // namespace

namespace cloth {
int net_last_cuda_error() { return g_net_cuda; }
void net_record_cuda_error(int e) { g_net_cuda = e; }
}

extern "C" {

int net_workspace_size(size_t* bytes)
{
    if (!bytes) return CLOTH_EINVAL;
    *bytes = net_layout().total;
    return CLOTH_OK;
}

int net_create(cloth_net** out, int32_t precision, const float* h_blob, void* d_workspace, size_t bytes, void* stream)
{
    if (!out || !h_blob || !d_workspace) return CLOTH_EINVAL;
    if (precision != CLOTH_NET_FP32 && precision != CLOTH_NET_BF16) return CLOTH_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256) return CLOTH_EINVAL;
    for (int i = 0; i < kBlob; ++i)
        if (!std::isfinite(h_blob[i])) return CLOTH_EINVAL;
    const NetLayout L = net_layout();
    if (bytes < L.total) return CLOTH_ENOMEM;
    int rc = ensure_init();
    if (rc) return rc;
    cloth_net* n = new (std::nothrow) cloth_net;
    if (!n) return CLOTH_ENOMEM;
    n->precision = precision;
    n->ws = static_cast<char*>(d_workspace);
    n->L = L;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->d_w(), h_blob, sizeof(float) * kBlob, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->d_status(), 0, 64, s);
    if (e == cudaSuccess) e = launch_pack_bf16(n->d_w(), n->d_pack(), s);
    if (e == cudaSuccess) e = launch_pack_comp(n->d_w(), n->d_comp(), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete n;
        return net_cuda_fail(e);
    }
    *out = n;
    return CLOTH_OK;
}

int net_set_weights(cloth_net* n, const float* d_blob, void* stream)
{
    if (!n || !d_blob) return CLOTH_EINVAL;
    NCK(cudaMemcpyAsync(n->d_w(), d_blob, sizeof(float) * kBlob, cudaMemcpyDeviceToDevice,
                        static_cast<cudaStream_t>(stream)));
    NCK(launch_pack_bf16(n->d_w(), n->d_pack(), static_cast<cudaStream_t>(stream)));
    NCK(launch_pack_comp(n->d_w(), n->d_comp(), static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

int net_get_weights(const cloth_net* n, float* d_blob, void* stream)
{
    if (!n || !d_blob) return CLOTH_EINVAL;
    NCK(cudaMemcpyAsync(d_blob, n->d_w(), sizeof(float) * kBlob, cudaMemcpyDeviceToDevice,
                        static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

int net_saved_size(int32_t N, int32_t H, int32_t W, size_t* bytes)
{
    if (!bytes || !dims_ok(N, H, W)) return CLOTH_EINVAL;
    *bytes = sizeof(float) * (size_t)kSavedPerNode * N * H * W;
    return CLOTH_OK;
}

int net_forward(cloth_net* n, const float* d_z, float* d_a, int32_t N, int32_t H, int32_t W, float* d_saved,
                void* stream)
{
    if (!n || !d_z || !d_a || !dims_ok(N, H, W)) return CLOTH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n->precision == CLOTH_NET_BF16) {
        if (d_saved) return CLOTH_EINVAL;   // the fused tensor-core kernel keeps nothing
        NCK(launch_net_tc_forward(n->d_pack(), n->d_w(), d_z, d_a, N, H, W, n->d_status(), n->sm_count, s));
        return CLOTH_OK;
    }
    if (!d_saved) return CLOTH_EINVAL;   // the FP32 path keeps its layer outputs there
    const int64_t NHW = (int64_t)N * H * W;
    NetFwdArgs f{};
    f.src.z = d_z;
    f.w = n->d_w();
    f.t1 = d_saved + kSavT1 * NHW;
    f.t2 = d_saved + kSavT2 * NHW;
    f.s = d_saved + kSavS * NHW;
    f.a = d_a;
    f.N = N; f.H = H; f.W = W;
    f.status = n->d_status();
    NCK(launch_net_forward_simt(f, s));
    return CLOTH_OK;
}

int net_backward(cloth_net* n, const float* d_z, float* d_saved, const float* d_grad_a, float* d_grad_z,
                 float* d_grad_w, int32_t N, int32_t H, int32_t W, void* stream)
{
    if (!n || !d_z || !d_saved || !d_grad_a || !d_grad_w || !dims_ok(N, H, W)) return CLOTH_EINVAL;
    if (n->precision != CLOTH_NET_FP32) return CLOTH_EUNSUPPORTED;
    NCK(launch_net_backward_simt(n->d_w(), d_z, d_saved, d_grad_a, d_grad_z, n->d_part(), d_grad_w, N, H, W,
                                 n->d_status(), static_cast<cudaStream_t>(stream)));
    return CLOTH_OK;
}

void net_destroy(cloth_net* n) { delete n; }

}  // extern "C"
