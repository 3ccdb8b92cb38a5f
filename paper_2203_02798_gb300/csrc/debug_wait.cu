// debug_wait.cu -- failure-detection check for the bounded device waits.
//
// One block waits, with the same tc::mbar_wait the tensor-core pipelines
// use, on an mbarrier that nothing arrives on.  The wait must give up after
// its limit; the kernel then sets the context's TIMEOUT flag and returns, so
// the host sees LSK_ERR_TIMEOUT at the next lsk_sync and the context remains
// usable.  No GPU fault is involved: the wait is bounded by %globaltimer.
#include "tc_common.cuh"

namespace {

__global__ void wait_timeout_kernel(uint64_t limit_ns, int* flag) {
    __shared__ uint64_t bar;
    __shared__ int abort;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);   // expects one arrival; none comes
        abort = 0;
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = tc::mbar_wait(&bar, 0, reinterpret_cast<volatile int*>(&abort), limit_ns);
        if (!ok) set_flag(flag, LSK_FLAG_TIMEOUT);
    }
    __syncthreads();
}

}  // namespace

cudaError_t debug_wait_timeout_launch(int64_t limit_us, int* flag, cudaStream_t st) {
    wait_timeout_kernel<<<1, 32, 0, st>>>((uint64_t)limit_us * 1000ull, flag);
    return cudaGetLastError();
}
