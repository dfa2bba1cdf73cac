// given.cu -- the given-P mode: the unique L and D of P^T A P = L D L^T for a
// pivot order and block structure supplied by the caller (for instance those
// of Algorithm 2/3, whose order differs from Algorithm 4's: Section 4 versus
// Section 5).
//
// For odd p, L and D are unique once P and the block structure are fixed: a
// 1x1 pivot is the Schur diagonal entry, and a 2x2 block [[0, x], [x, y]] has
// the one congruence [[1, 0], [y/(2x), 1]] [[0, x], [x, 0]] [[1, y/(2x)], [0, 1]].
// For p = 2 the block keeps [[0, x], [x, y]] and in-block entry 0.  A
// structure that fits A has, at every 1x1 position, a non-zero Schur
// diagonal; at every 2x2 start a zero diagonal and a non-zero next entry; and
// a zero Schur complement after the rank.  Algorithm 4's lexicographic search
// run on S = P^T A P then takes exactly the identity order with the same
// blocks, so the factorisation of S is the answer.  Hence: S is gathered in
// the ingest pass (factor_core with the order), factored by the same GPU
// path, and checked: order = identity, block starts and rank as supplied;
// anything else means the structure does not fit A (LDLT_ERR_INCONSISTENT).
#include <cstdint>

#include "../../include/ldlt_rpm.h"
#include "ldlt_internal.cuh"

namespace {

size_t r256(size_t x) { return (x + 255) & ~(size_t)255; }

struct GivenExtra {
    size_t psave, emark, cnt, flags, total;
};

GivenExtra given_extra(int64_t n)
{
    GivenExtra g;
    g.psave = 0;
    g.emark = g.psave + r256((size_t)n * 4);
    g.cnt = g.emark + r256((size_t)n);
    g.flags = g.cnt + r256((size_t)n * 4);
    g.total = g.flags + 256;  // int bad, int pad, int64 rank
    return g;
}

// save the supplied order, block starts and rank; count each index of perm
__global__ void gv_prep_kernel(int64_t n, const int32_t *perm, const uint32_t *e, const int64_t *rank,
                               int32_t *psave, uint8_t *emark, int *cnt, int *flags)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) reinterpret_cast<int64_t *>(flags)[1] = *rank;
    if (k >= n) return;
    const int32_t v = perm[k];
    psave[k] = v;
    emark[k] = e[k] != 0u;
    if (v >= 0 && v < n) atomicAdd(cnt + v, 1);
    else atomicExch(flags, 1);
}

// every index exactly once
__global__ void gv_perm_check_kernel(int64_t n, const int *cnt, int *flags)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && cnt[k] != 1) atomicExch(flags, 1);
}

// compare the factorisation of P^T A P with the supplied structure and put the
// supplied order back as the output order
__global__ void gv_finish_kernel(int64_t n, int32_t *perm, const uint32_t *e, const int64_t *rank,
                                 const int32_t *psave, const uint8_t *emark, const int *flags, int32_t *status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool badperm = flags[0] != 0;  // reported alone: the order was not a permutation
    if (k == 0) {
        if (badperm) atomicCAS(status, 0, LDLT_ERR_ARG);
        else if (*rank != reinterpret_cast<const int64_t *>(flags)[1]) atomicCAS(status, 0, LDLT_ERR_INCONSISTENT);
    }
    if (k >= n) return;
    if (!badperm && (perm[k] != (int32_t)k || (uint8_t)(e[k] != 0u) != emark[k]))
        atomicCAS(status, 0, LDLT_ERR_INCONSISTENT);
    perm[k] = psave[k];
}

}  // namespace

extern "C" int ldlt_rpm_given_workspace_bytes(int64_t n, uint32_t p, int path, size_t *bytes)
{
    if (!bytes) return LDLT_ERR_ARG;
    size_t fb = 0;
    const int rc = ldlt_rpm_workspace_bytes(n, p, path, &fb);
    if (rc != LDLT_OK) return rc;
    *bytes = r256(fb) + given_extra(n).total;
    return LDLT_OK;
}

extern "C" int ldlt_rpm_factor_given(int64_t n, uint32_t p, uint32_t *A, int64_t lda, int32_t *perm,
                                     uint32_t *e, int64_t *rank, int32_t *status, int path, void *ws,
                                     size_t ws_bytes, void *stream)
{
    size_t fb = 0, need = 0;
    int rc = ldlt_rpm_workspace_bytes(n, p, path, &fb);
    if (rc != LDLT_OK) return rc;
    if (!rank || !status) return LDLT_ERR_ARG;
    if (n > 0 && (!A || !perm || !e || lda < n)) return LDLT_ERR_ARG;
    rc = ldlt_rpm_given_workspace_bytes(n, p, path, &need);
    if (rc != LDLT_OK) return rc;
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255) != 0) return LDLT_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) return factor_core(n, p, A, lda, perm, e, rank, status, path, ws, fb, stream, nullptr, nullptr);
    const GivenExtra g = given_extra(n);
    uint8_t *x = (uint8_t *)ws + r256(fb);
    int32_t *psave = (int32_t *)(x + g.psave);
    uint8_t *emark = x + g.emark;
    int *cnt = (int *)(x + g.cnt);
    int *flags = (int *)(x + g.flags);
    if (cudaMemsetAsync(cnt, 0, (size_t)n * 4, st) != cudaSuccess) return LDLT_ERR_CUDA;
    if (cudaMemsetAsync(flags, 0, 16, st) != cudaSuccess) return LDLT_ERR_CUDA;
    const unsigned gk = (unsigned)((n + 255) / 256);
    gv_prep_kernel<<<gk, 256, 0, st>>>(n, perm, e, rank, psave, emark, cnt, flags);
    gv_perm_check_kernel<<<gk, 256, 0, st>>>(n, cnt, flags);
    if (cudaGetLastError() != cudaSuccess) return LDLT_ERR_CUDA;
    rc = factor_core(n, p, A, lda, perm, e, rank, status, path, ws, fb, stream, psave, flags);
    if (rc != LDLT_OK) return rc;
    gv_finish_kernel<<<gk, 256, 0, st>>>(n, perm, e, rank, psave, emark, flags, status);
    return cudaGetLastError() == cudaSuccess ? LDLT_OK : LDLT_ERR_CUDA;
}
