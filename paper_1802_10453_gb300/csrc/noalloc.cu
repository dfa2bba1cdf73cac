// noalloc.cu -- ldlt_rpm_factor_noalloc: the factorisation with its scratch in
// a fixed device array that belongs to the library, for callers that must not
// allocate device memory while they run (the contract is in include/ldlt_rpm.h).
//
// The array lives in this translation unit only, so its memory is reserved
// when this module is loaded -- under CUDA's default lazy module loading, at
// the first call -- and not by every program that opens the library.  The kernels are the ones ldlt_rpm_factor
// launches; only the origin of the scratch pointer differs.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ldlt_rpm.h"

static __device__ __align__(256) unsigned char g_noalloc_ws[LDLT_NOALLOC_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_ws on the current device, looked up once per
// device; nullptr if the lookup fails.
void *noalloc_scratch(int dev)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_ws) != cudaSuccess) {
            (void)cudaGetLastError();  // leave no pending error behind for the caller
            return nullptr;
        }
        g_noalloc_ptr[dev] = ptr;
    }
    return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" int ldlt_rpm_factor_noalloc(int64_t n, uint32_t p, uint32_t *A, int64_t lda, int32_t *perm,
                                       uint32_t *e, int64_t *rank, int32_t *status, int path,
                                       void *stream)
{
    size_t need = 0;
    const int rc = ldlt_rpm_workspace_bytes(n, p, path, &need);  // n, p and path checks
    if (rc != LDLT_OK) return rc;
    if (n > LDLT_NOALLOC_MAX_N || need > sizeof(g_noalloc_ws)) return LDLT_ERR_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDLT_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LDLT_ERR_NO_DEVICE;
    void *ws = noalloc_scratch(dev);
    if (!ws) return LDLT_ERR_CUDA;
    return ldlt_rpm_factor(n, p, A, lda, perm, e, rank, status, path, ws, sizeof(g_noalloc_ws), stream);
}
