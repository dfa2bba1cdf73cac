// strict_char2.cu -- Section 2.2 (Antitriangular decomposition): turn the
// relaxed 2x2 blocks [[0, c], [c, d]] (d != 0) of a characteristic-2
// factorisation P^T A P = L D L^T into pairs of 1x1 pivots, in place on the
// output of ldlt_rpm_factor (L strictly below the diagonal of A, D on it, 2x2
// block starts in e, pivot order in perm).
//
// Over F_2 every non-zero is 1, so for a block (k, k+1) with c = d = 1:
//   1. the block is invariant under [[1, 0], [l, 1]] congruence mod 2, so L's
//      in-block entry l is folded into column k (column k += l * column k+1);
//   2. [[0, 1], [1, 1]] = J [[1, 0], [1, 1]] diag(1, 1) [[1, 1], [0, 1]] J, so
//      the positions k, k+1 swap in perm, rows and columns k, k+1 of L swap,
//      then column k += column k+1, the new in-block entry is 1 and D's block
//      becomes diag(1, 1).
// Blocks with d = 0 are antidiagonal already.  Cost: one pass over the rows,
// O(n) per row.  The rank profile matrix is no longer P Psi P^T afterwards.
#include <cstdint>

#include "../../include/ldlt_rpm.h"
#include "ldlt_internal.cuh"

namespace {

constexpr uint32_t MARK = 2u;  // e[k] while block (k, k+1) is being transformed

// e[k] = MARK for every block (k, k+1) with a non-zero corner d = A[k+1][k+1]
__global__ void char2_mark_kernel(int64_t n, const uint32_t *A, int64_t lda, uint32_t *e)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k + 1 >= n) return;
    if (e[k] != 0u && A[(k + 1) * lda + k + 1] != 0u) e[k] = MARK;
}

// new values of a marked column pair (j, j+1) of one row, from that row's
// old values (r0, r1) and the block's in-block entry l = A[j+1][j]
__device__ __forceinline__ void char2_pair(uint32_t r0, uint32_t r1, uint32_t l, uint32_t &n0, uint32_t &n1)
{
    const uint32_t f0 = r0 ^ (l & r1);  // step 1: column j += l column j+1
    n0 = r1 ^ f0;                       // step 2: swap the columns, then column j += column j+1
    n1 = f0;
}

// One CTA per row t.  A row outside the marked blocks keeps its position and
// only its marked column pairs left of t change.  The first row k of a marked
// block takes the pair of rows (k, k+1): new row k is old row k+1 and new row
// k+1 is old row k, both transformed (columns < k).
__global__ void char2_rows_kernel(int64_t n, uint32_t *A, int64_t lda, const uint32_t *e)
{
    const int64_t t = blockIdx.x;
    if (t >= n) return;
    if (t >= 1 && e[t - 1] == MARK) return;  // second row of a marked block: done by row t-1
    uint32_t *rt = A + t * lda;
    if (t + 1 < n && e[t] == MARK) {
        uint32_t *rn = rt + lda;
        for (int64_t j = threadIdx.x; j < t; j += blockDim.x) {
            if (j >= 1 && e[j - 1] == MARK) continue;  // second column of a pair: done at j-1
            if (e[j] == MARK) {                       // pair (j, j+1), j + 1 < t
                const uint32_t l = A[(j + 1) * lda + j];
                const uint32_t a0 = rt[j], a1 = rt[j + 1], b0 = rn[j], b1 = rn[j + 1];
                uint32_t x0, x1, y0, y1;
                char2_pair(b0, b1, l, x0, x1);
                char2_pair(a0, a1, l, y0, y1);
                rt[j] = x0; rt[j + 1] = x1;
                rn[j] = y0; rn[j + 1] = y1;
            } else {
                const uint32_t a = rt[j], b = rn[j];
                rt[j] = b;
                rn[j] = a;
            }
        }
        return;
    }
    for (int64_t j = threadIdx.x; j + 1 < t; j += blockDim.x) {
        if (e[j] != MARK) continue;
        const uint32_t l = A[(j + 1) * lda + j];
        uint32_t n0, n1;
        char2_pair(rt[j], rt[j + 1], l, n0, n1);
        rt[j] = n0;
        rt[j + 1] = n1;
    }
}

// per marked block: positions swap, D's block becomes diag(1, 1), the new
// in-block entry of L is 1, the block start mark is cleared
__global__ void char2_finish_kernel(int64_t n, uint32_t *A, int64_t lda, int32_t *perm, uint32_t *e)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k + 1 >= n || e[k] != MARK) return;
    const int32_t pk = perm[k];
    perm[k] = perm[k + 1];
    perm[k + 1] = pk;
    A[k * lda + k] = 1u;
    A[(k + 1) * lda + k + 1] = 1u;
    A[(k + 1) * lda + k] = 1u;
    e[k] = 0u;
}

}  // namespace

extern "C" int ldlt_rpm_strict(int64_t n, uint32_t p, uint32_t *A, int64_t lda, int32_t *perm, uint32_t *e,
                               void *stream)
{
    size_t tmp = 0;
    const int rc = ldlt_rpm_workspace_bytes(1, p, LDLT_PATH_TC, &tmp);  // p prime, in range
    if (rc != LDLT_OK) return rc;
    if (n < 0) return LDLT_ERR_ARG;
    if (n > 0 && (!A || !perm || !e || lda < n)) return LDLT_ERR_ARG;
    if (p != 2 || n < 2) return LDLT_OK;  // odd p: Algorithm 4's blocks are antidiagonal already
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned gk = (unsigned)((n + 255) / 256);
    char2_mark_kernel<<<gk, 256, 0, st>>>(n, A, lda, e);
    char2_rows_kernel<<<(unsigned)n, 128, 0, st>>>(n, A, lda, e);
    char2_finish_kernel<<<gk, 256, 0, st>>>(n, A, lda, perm, e);
    return cudaGetLastError() == cudaSuccess ? LDLT_OK : LDLT_ERR_CUDA;
}
