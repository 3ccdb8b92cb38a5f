// noalloc.cu -- a CountSketch entry point that allocates no device memory.
//
// lsk_cs_sketch needs scratch space (bucket counts, bucket offsets and fill
// cursors, and the bucket-sorted row permutation) and takes it from a
// context workspace that grows with cudaMallocAsync.  Some callers cannot let
// a library allocate: applications that hand all device memory to their own
// pool allocator (so a foreign cudaMalloc can fail or break their budget),
// and latency-critical loops where cudaMalloc / cudaFree may synchronise the
// device.  lsk_cs_sketch_noalloc serves them: it runs the same kernels, but
// its scratch lives in one fixed-size array in device global memory, so a
// call allocates nothing.
//
// The CUDA runtime loads a library's device code lazily: the array (and the
// CountSketch kernels' code) is placed on a device when the first call on
// that device looks the array up.  That first call is therefore the one that
// takes device memory (12 MiB plus the code); a caller that must not see a
// later allocation makes one call during its set-up, before any stream
// capture.  Every later call on that device allocates nothing.
//
// The array is shared by every call in the process, so calls whose GPU work
// overlaps (two streams, two host threads) race on it; serialise them.  It
// keeps whatever the previous call left: the bucket counts are cleared at
// the start of every call, every other piece is overwritten before it is read.
#include "lsk_internal.cuh"

#include <mutex>

namespace {

constexpr size_t kNoallocScratchBytes = 12u << 20;  // 12 MiB on each device that has made a call, until exit

// Device-side scratch.  Host code must not pass this name to a kernel (on the
// host it is only a stand-in symbol); the device address comes from
// cudaGetSymbolAddress, once per device, below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct DeviceSlot {
    void* scratch = nullptr;
    int sm_count = 0;
    bool ready = false;
};
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
DeviceSlot g_slots[kMaxDevices];

int check_args(const lsk_mat* A, int64_t r, const float* SA) {
    if (!A || !SA) return LSK_ERR_INVALID_ARG;
    if (A->dtype != LSK_F32) return LSK_ERR_UNSUPPORTED;
    if (A->n < 0 || A->d < 1) return LSK_ERR_INVALID_ARG;
    if (r < 1) return LSK_ERR_INVALID_ARG;
    if (A->kind == LSK_DENSE) {
        if (A->ld < A->d || (A->n > 0 && !A->values)) return LSK_ERR_INVALID_ARG;
    } else if (A->kind == LSK_CSR) {
        if (!A->rowptr || A->nnz < 0 || (A->nnz > 0 && (!A->colidx || !A->values))) return LSK_ERR_INVALID_ARG;
        if (A->d > 51200) return LSK_ERR_UNSUPPORTED;
    } else {
        return LSK_ERR_INVALID_ARG;
    }
    // the fixed capacity: rows, buckets, and the scratch they need together
    if (A->n > LSK_NOALLOC_MAX_ROWS || r > LSK_NOALLOC_MAX_BUCKETS) return LSK_ERR_UNSUPPORTED;
    if (cs_workspace_bytes_atomic(A->n, r) > kNoallocScratchBytes) return LSK_ERR_UNSUPPORTED;
    return LSK_OK;
}

// Resolve the scratch array's device address for the current device (first
// call on that device only).
int device_slot(DeviceSlot** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LSK_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSlot& s = g_slots[dev];
    if (!s.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return LSK_ERR_CUDA;
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return LSK_ERR_CUDA;
        }
        s.scratch = p;
        s.sm_count = sms;
        s.ready = true;
    }
    *out = &s;
    return LSK_OK;
}

}  // namespace

extern "C" int lsk_cs_sketch_noalloc(const lsk_mat* A, int64_t r, uint64_t seed, float* SA, void* stream) {
    int rc = check_args(A, r, SA);
    if (rc) return rc;
    DeviceSlot* slot = nullptr;
    rc = device_slot(&slot);
    if (rc) return rc;
    // CSR entries out of range are skipped by the kernels; with no context
    // there is no flag to report them through (flag = NULL).
    // the atomic form, whose scratch the fixed capacity is sized for
    cudaError_t e = cs_launch(A, r, seed, SA, slot->scratch, nullptr, slot->sm_count, (cudaStream_t)stream, 0, false,
                              nullptr, nullptr, false);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? LSK_OK : LSK_ERR_CUDA;
}
