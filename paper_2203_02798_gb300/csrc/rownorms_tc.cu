// rownorms_tc.cu -- tensor-core (tcgen05) path of the dense row-norm GEMM.
#include "lsk_internal.cuh"

bool rownorms_tc_supported(const lsk_mat*, int64_t) { return false; }
cudaError_t rownorms_tc_launch(const lsk_mat*, const float*, int64_t, float, float, int, float*, void*, int,
                               cudaStream_t) {
    return cudaErrorNotSupported;
}
