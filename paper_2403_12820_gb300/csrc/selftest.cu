// Self-test of the bounded-wait path every tensor-core wait takes: one warp
// initialises an mbarrier that nothing will ever complete, polls it a
// bounded number of times, and on running out sets the timeout bit of the
// status word and returns, the same way net_tc_kernel leaves a wait that
// ran out.  Nothing spins without a bound and nothing traps.
#include "cloth_internal.cuh"
#include "tc_ptx.cuh"

namespace cloth {
namespace {

__global__ void wait_timeout_kernel(int32_t* status, uint32_t polls)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = tc::smem_u32(&bar);
    if (threadIdx.x == 0) {
        tc::mbar_init(b, 1);   // one arrival expected; none comes
        tc::fence_mbar_init();
    }
    __syncwarp();
    const bool done = tc::mbar_wait(b, 0u, polls);
    if (!__any_sync(0xffffffffu, done) && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

}  // namespace

cudaError_t launch_wait_timeout_selftest(int32_t* status, uint32_t polls, cudaStream_t s)
{
    wait_timeout_kernel<<<1, 32, 0, s>>>(status, polls);
    return cudaGetLastError();
}

}  // namespace cloth
