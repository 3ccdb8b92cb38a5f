// gauss_tc.cu -- tensor-core (tcgen05) path of the Gaussian stage (BF16).
#include "lsk_internal.cuh"

bool gauss_tc_supported(int64_t, int64_t, int64_t) { return false; }
size_t gauss_tc_workspace_bytes(int64_t, int64_t, int64_t, int) { return 0; }
cudaError_t gauss_tc_launch(const float*, int64_t, int64_t, int64_t, uint64_t, float*, void*, int,
                            cudaStream_t) {
    return cudaErrorNotSupported;
}
