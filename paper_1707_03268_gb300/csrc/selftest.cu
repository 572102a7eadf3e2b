// Failure-detection self-test: a kernel whose mbarrier wait can never complete (no thread arrives). The wait is the
// bounded one every tensor-core kernel uses: it gives up after its limit, raises the context's device error flag and
// returns, so the kernel exits cleanly and the host reads the expiry as ERR_TIMEOUT. Nothing faults or hangs.
#include "internal.h"
#include "tc_ptx.h"

namespace tdpm {
namespace {

__global__ void bounded_wait_probe_kernel(int *err)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(b, 0, err);  // no arrival ever comes: expires
}

}  // namespace

cudaError_t launch_bounded_wait_probe(int *d_err, cudaStream_t s)
{
    note_launches(1);
    bounded_wait_probe_kernel<<<1, 32, 0, s>>>(d_err);
    return cudaGetLastError();
}

}  // namespace tdpm
