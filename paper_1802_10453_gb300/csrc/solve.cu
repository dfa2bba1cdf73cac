// solve.cu -- A X = B from the factorisation P^T A P = L D L^T (the use the
// paper's Section 1 gives for a symmetric triangular factorisation: solving
// symmetric systems).  With the factor stored as ldlt_rpm_factor leaves it (L
// strictly below the diagonal of A, D on it and in e, pivot order in perm):
//   Z = P^T B                       gather rows
//   L Z' = Z                        forward substitution, unit diagonal
//   D W = Z'                        1x1 pivots, 2x2 blocks [[0, x], [x, y]];
//                                   rows k >= rank: consistent only if 0
//   L^T V = W                       backward substitution
//   X = P V                         scatter rows
// The triangular solves run in blocks of SB rows: one CTA solves the diagonal
// block (staged in shared memory; one warp per right-hand-side column, the
// block's rows in sequence, each row's dot split over the lanes), then every
// remaining row takes the block's contribution (one thread per (row, column),
// SB multiply-adds with one reduction).  Bounded work, no
// inter-CTA waits; block steps are ordered by the stream.
#include <cstdint>

#include "../../include/ldlt_rpm.h"
#include "ldlt_internal.cuh"

namespace {

constexpr int SB = 64;

__global__ void sv_gather_kernel(int64_t n, int64_t nrhs, const int32_t *perm, const uint32_t *B, int64_t ldb,
                                 uint32_t *Z, FieldP f)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    const int64_t k = idx / nrhs, c = idx - k * nrhs;
    const uint32_t v = B[(int64_t)perm[k] * ldb + c];
    Z[idx] = v >= f.p ? v % f.p : v;
}

// The diagonal block of L (rows and columns [b0, b1)) staged in shared memory
// (row stride SB + 1: conflict-free column reads for the transposed solve).
__device__ __forceinline__ void sv_stage_block(uint32_t (*Lb)[SB + 1], int64_t b0, int nb, const uint32_t *A,
                                               int64_t lda)
{
    for (int q = threadIdx.x; q < SB * SB; q += blockDim.x) {
        const int r = q / SB, c = q % SB;
        Lb[r][c] = (r < nb && c < nb) ? A[(b0 + r) * lda + b0 + c] : 0u;
    }
    __syncthreads();
}

// sum over the warp of per-lane residues, mod p (every lane gets the result)
__device__ __forceinline__ uint32_t sv_warp_sum(uint32_t v, const FieldP &f)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fp_add(v, __shfl_xor_sync(0xffffffffu, v, o), f);
    return v;
}

// rows [b0, b1): Z[i] -= sum_{b0 <= j < i} L[i][j] Z[j].  One warp per
// right-hand-side column: lane l holds rows b0 + l and b0 + 32 + l; the dot of
// row i is split over the lanes and summed by shuffles.
__global__ void sv_fwd_diag_kernel(int64_t b0, int64_t b1, const uint32_t *A, int64_t lda, uint32_t *Z,
                                   int64_t nrhs, FieldP f)
{
    __shared__ uint32_t Lb[SB][SB + 1];
    const int nb = (int)(b1 - b0);
    sv_stage_block(Lb, b0, nb, A, lda);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t c = warp; c < nrhs; c += nw) {
        uint32_t z0 = lane < nb ? Z[(b0 + lane) * nrhs + c] : 0u;
        uint32_t z1 = lane + 32 < nb ? Z[(b0 + 32 + lane) * nrhs + c] : 0u;
        for (int i = 1; i < nb; ++i) {
            uint64_t acc = 0;
            if (lane < i) fp_mac(acc, Lb[i][lane], z0, f);
            if (lane + 32 < i) fp_mac(acc, Lb[i][lane + 32], z1, f);
            const uint32_t s = sv_warp_sum(fp_reduce64(acc, f), f);
            if (i == lane) z0 = fp_sub(z0, s, f);
            if (i == lane + 32) z1 = fp_sub(z1, s, f);
        }
        if (lane < nb) Z[(b0 + lane) * nrhs + c] = z0;
        if (lane + 32 < nb) Z[(b0 + 32 + lane) * nrhs + c] = z1;
    }
}

// rows i >= b1: Z[i] -= sum_{b0 <= j < b1} L[i][j] Z[j]
__global__ void sv_fwd_update_kernel(int64_t n, int64_t b0, int64_t b1, const uint32_t *A, int64_t lda,
                                     uint32_t *Z, int64_t nrhs, FieldP f)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = b1 + idx / nrhs, c = idx % nrhs;
    if (i >= n) return;
    const uint32_t *Li = A + i * lda;
    uint64_t acc = 0;
    for (int64_t j = b0; j < b1; ++j) fp_mac(acc, Li[j], Z[j * nrhs + c], f);
    Z[i * nrhs + c] = fp_sub(Z[i * nrhs + c], fp_reduce64(acc, f), f);
}

// D W = Z in place; rows k >= rank must be zero for a consistent system
__global__ void sv_dsolve_kernel(int64_t n, const uint32_t *A, int64_t lda, const uint32_t *e,
                                 const int64_t *rank, uint32_t *Z, int64_t nrhs, FieldP f, int32_t *status)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    const int64_t k = idx / nrhs, c = idx - k * nrhs;
    const int64_t r = *rank;
    if (k >= r) {
        if (Z[idx] != 0u) atomicExch(status, LDLT_ERR_INCONSISTENT);
        Z[idx] = 0u;
        return;
    }
    if (k >= 1 && e[k - 1] != 0u) return;  // second row of a 2x2 block: done by row k-1
    if (e[k] != 0u) {
        // [[0, x], [x, y]] [w0, w1]^T = [z0, z1]^T: w1 = z0 / x, w0 = (z1 - y w1) / x
        const uint32_t x = e[k], y = A[(k + 1) * lda + k + 1];
        const uint32_t ix = fp_inv(x, f);
        const uint32_t w1 = fp_mul(Z[idx], ix, f);
        const uint32_t w0 = fp_mul(fp_sub(Z[idx + nrhs], fp_mul(y, w1, f), f), ix, f);
        Z[idx] = w0;
        Z[idx + nrhs] = w1;
    } else {
        Z[idx] = fp_mul(Z[idx], fp_inv(A[k * lda + k], f), f);
    }
}

// rows [b0, b1) from the last: Z[i] -= sum_{i < j < b1} L[j][i] Z[j] (warp per column)
__global__ void sv_bwd_diag_kernel(int64_t b0, int64_t b1, const uint32_t *A, int64_t lda, uint32_t *Z,
                                   int64_t nrhs, FieldP f)
{
    __shared__ uint32_t Lb[SB][SB + 1];
    const int nb = (int)(b1 - b0);
    sv_stage_block(Lb, b0, nb, A, lda);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t c = warp; c < nrhs; c += nw) {
        uint32_t z0 = lane < nb ? Z[(b0 + lane) * nrhs + c] : 0u;
        uint32_t z1 = lane + 32 < nb ? Z[(b0 + 32 + lane) * nrhs + c] : 0u;
        for (int i = nb - 2; i >= 0; --i) {
            uint64_t acc = 0;
            if (lane > i && lane < nb) fp_mac(acc, Lb[lane][i], z0, f);
            if (lane + 32 > i && lane + 32 < nb) fp_mac(acc, Lb[lane + 32][i], z1, f);
            const uint32_t s = sv_warp_sum(fp_reduce64(acc, f), f);
            if (i == lane) z0 = fp_sub(z0, s, f);
            if (i == lane + 32) z1 = fp_sub(z1, s, f);
        }
        if (lane < nb) Z[(b0 + lane) * nrhs + c] = z0;
        if (lane + 32 < nb) Z[(b0 + 32 + lane) * nrhs + c] = z1;
    }
}

// rows i < b0: Z[i] -= sum_{b0 <= j < b1} L[j][i] Z[j]
__global__ void sv_bwd_update_kernel(int64_t b0, int64_t b1, const uint32_t *A, int64_t lda, uint32_t *Z,
                                     int64_t nrhs, FieldP f)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = idx / nrhs, c = idx % nrhs;
    if (i >= b0) return;
    uint64_t acc = 0;
    for (int64_t j = b0; j < b1; ++j) fp_mac(acc, A[j * lda + i], Z[j * nrhs + c], f);
    Z[i * nrhs + c] = fp_sub(Z[i * nrhs + c], fp_reduce64(acc, f), f);
}

__global__ void sv_scatter_kernel(int64_t n, int64_t nrhs, const int32_t *perm, const uint32_t *Z, uint32_t *X,
                                  int64_t ldx)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    const int64_t k = idx / nrhs, c = idx - k * nrhs;
    X[(int64_t)perm[k] * ldx + c] = Z[idx];
}

unsigned nblk(int64_t work, int t) { return (unsigned)((work + t - 1) / t); }

}  // namespace

extern "C" int ldlt_rpm_solve(int64_t n, uint32_t p, const uint32_t *A, int64_t lda, const int32_t *perm,
                              const uint32_t *e, const int64_t *rank, const uint32_t *B, int64_t ldb, int64_t nrhs,
                              uint32_t *X, int64_t ldx, int32_t *status, void *ws, size_t ws_bytes, void *stream)
{
    size_t tmp = 0;
    const int rc = ldlt_rpm_workspace_bytes(1, p, LDLT_PATH_TC, &tmp);  // p prime, in range
    if (rc != LDLT_OK) return rc;
    if (n < 0 || nrhs < 0 || !status) return LDLT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return LDLT_ERR_CUDA;
    if (n == 0 || nrhs == 0) return LDLT_OK;
    if (!A || !perm || !e || !rank || !B || !X || lda < n || ldb < nrhs || ldx < nrhs) return LDLT_ERR_ARG;
    if (!ws || ws_bytes < (size_t)n * (size_t)nrhs * 4) return LDLT_ERR_WORKSPACE;
    const FieldP f = make_field(p);
    uint32_t *Z = (uint32_t *)ws;
    const int T = 256;
    sv_gather_kernel<<<nblk(n * nrhs, T), T, 0, st>>>(n, nrhs, perm, B, ldb, Z, f);
    for (int64_t b0 = 0; b0 < n; b0 += SB) {
        const int64_t b1 = b0 + SB < n ? b0 + SB : n;
        sv_fwd_diag_kernel<<<1, T, 0, st>>>(b0, b1, A, lda, Z, nrhs, f);
        if (b1 < n) sv_fwd_update_kernel<<<nblk((n - b1) * nrhs, T), T, 0, st>>>(n, b0, b1, A, lda, Z, nrhs, f);
    }
    sv_dsolve_kernel<<<nblk(n * nrhs, T), T, 0, st>>>(n, A, lda, e, rank, Z, nrhs, f, status);
    for (int64_t b1 = n; b1 > 0; b1 -= (b1 % SB ? b1 % SB : SB)) {
        const int64_t b0 = b1 - (b1 % SB ? b1 % SB : SB);
        sv_bwd_diag_kernel<<<1, T, 0, st>>>(b0, b1, A, lda, Z, nrhs, f);
        if (b0 > 0) sv_bwd_update_kernel<<<nblk(b0 * nrhs, T), T, 0, st>>>(b0, b1, A, lda, Z, nrhs, f);
    }
    sv_scatter_kernel<<<nblk(n * nrhs, T), T, 0, st>>>(n, nrhs, perm, Z, X, ldx);
    return cudaGetLastError() == cudaSuccess ? LDLT_OK : LDLT_ERR_CUDA;
}
