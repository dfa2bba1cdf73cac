// noalloc.cu -- ldlt_rpm_factor_noalloc: the factorisation with its scratch in
// a fixed device array that belongs to the library, for callers that must not
// allocate device memory while they run (the contract is in include/ldlt_rpm.h).
//
// The array lives in this translation unit only, so its memory is reserved
// when this module is loaded -- under CUDA's default lazy module loading, at
// the first call -- and not by every program that opens the library.  The kernels are the ones ldlt_rpm_factor
// launches; only the origin of the scratch pointer differs.
#include <cuda_runtime.h>

#include "../../include/ldlt_rpm.h"

static __device__ __align__(256) unsigned char g_noalloc_ws[LDLT_NOALLOC_BYTES];

namespace {

// Device address of g_noalloc_ws on the current device, looked up on every
// call (the lookup allocates nothing once the module is loaded, and a fresh
// lookup stays right after cudaDeviceReset or under another context);
// nullptr if the lookup fails.  A failed lookup clears only the error it
// raised itself: an error the caller had pending before the call stays.
void *noalloc_scratch()
{
    const bool clean_before = cudaPeekAtLastError() == cudaSuccess;
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_ws) != cudaSuccess) {
        if (clean_before) (void)cudaGetLastError();
        return nullptr;
    }
    return ptr;
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
    void *ws = noalloc_scratch();
    if (!ws) return LDLT_ERR_CUDA;
    return ldlt_rpm_factor(n, p, A, lda, perm, e, rank, status, path, ws, sizeof(g_noalloc_ws), stream);
}
