// Self-test of the bounded-wait failure path: one thread waits on an mbarrier
// that nothing arrives on.  The wait gives up after timeout_ns, records the
// time-out in the status word and the kernel returns normally.
#include "kernels.cuh"
#include "ptx.cuh"

namespace cpi {
namespace {

__global__ void wait_selftest_kernel(unsigned int* status, unsigned long long timeout_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, &abort_flag, status, timeout_ns);
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned int* status, unsigned long long timeout_ns,
                                 cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(status, timeout_ns);
    return cudaGetLastError();
}

}  // namespace cpi
