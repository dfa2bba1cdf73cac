// kernels_misc.cu -- the HBM-streaming steps around the pivot chain:
// ingest of A, storing the panel's L columns, compaction of the Schur
// complement when a panel took no pivot, the final symmetric permutation of L
// (PERM of Algorithm 2) and the rank profile matrix P Psi P^T (Section 2.1).
#include "ldlt_internal.cuh"

namespace {

// S[i][j] = A[i][j] mod p for j <= i (lower triangle only); idx = identity.
// One CTA per row.  When every row of A starts on a 16-byte boundary (vec),
// the row moves in 16-byte chunks (S rows are 256-byte aligned); the chunk
// that holds the diagonal is written element by element so nothing past it
// is read or written.
__device__ __forceinline__ uint32_t red_in(uint32_t v, const FieldP &f) { return v >= f.p ? v % f.p : v; }

__global__ void __launch_bounds__(256) ingest_kernel(const uint32_t *__restrict__ A, int64_t lda, int64_t n,
                                                     uint32_t *__restrict__ S, int64_t ldS,
                                                     int *__restrict__ idx, FieldP f, int vec)
{
    const int64_t i = blockIdx.x;
    if (i >= n) return;
    if (threadIdx.x == 0) idx[i] = (int)i;
    const uint32_t *src = A + i * lda;
    uint32_t *dst = S + i * ldS;
    const int64_t len = i + 1;
    int64_t j0 = 0;
    if (vec) {
        const int64_t nfull = len >> 2;  // chunks entirely at or left of the diagonal
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (int64_t c = threadIdx.x; c < nfull; c += blockDim.x) {
            uint4 v = __ldg(s4 + c);
            v.x = red_in(v.x, f); v.y = red_in(v.y, f); v.z = red_in(v.z, f); v.w = red_in(v.w, f);
            d4[c] = v;
        }
        j0 = nfull << 2;
    }
    for (int64_t j = j0 + threadIdx.x; j < len; j += blockDim.x) dst[j] = red_in(__ldg(src + j), f);
}

// The same for a supplied order: S[i][j] = A[perm[i]][perm[j]] mod p, read
// from A's lower triangle (the symmetric entry).  An index outside [0, n) sets
// *bad and is not read.
__global__ void ingest_perm_kernel(const uint32_t *__restrict__ A, int64_t lda, int64_t n,
                                   const int32_t *__restrict__ perm, uint32_t *__restrict__ S, int64_t ldS,
                                   int *__restrict__ idx, FieldP f, int *bad)
{
    const int64_t i = blockIdx.y;
    if (i >= n) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) idx[i] = (int)i;
    const int64_t a = perm[i];
    uint32_t *dst = S + i * ldS;
    const bool ra = a >= 0 && a < n;
    if (!ra && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(bad, 1);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= i;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = perm[j];
        uint32_t v = 0u;
        if (ra && b >= 0 && b < n) v = a >= b ? __ldg(A + a * lda + b) : __ldg(A + b * lda + a);
        else atomicExch(bad, 1);
        dst[j] = v >= f.p ? v % f.p : v;
    }
}

// Lw[idx[t]][col0 + j] = LpT[j][t]: transpose through shared memory so both
// the reads (along t) and the writes (along j) are coalesced.
__global__ void lw_scatter_kernel(const uint32_t *__restrict__ LpT, int64_t ldL, int m, int np,
                                  const int *__restrict__ idx, uint32_t *__restrict__ Lw,
                                  int64_t ldw, int col0)
{
    __shared__ uint32_t tile[32][33];
    const int t0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        int j = j0 + r, t = t0 + tx;
        if (j < np && t < m) tile[r][tx] = LpT[(int64_t)j * ldL + t];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        int t = t0 + r, j = j0 + tx;
        if (t < m && j < np) Lw[(int64_t)idx[t] * ldw + col0 + j] = tile[tx][r];
    }
}

// Snext[i][j] = S[sigma[i]][sigma[j]] for j <= i < m_next.
__global__ void compact_copy_kernel(const uint32_t *__restrict__ S, int64_t ldS,
                                    const int *__restrict__ sigma, int m_next,
                                    uint32_t *__restrict__ Snext)
{
    const int i = blockIdx.y;
    if (i >= m_next) return;
    const uint32_t *src = S + (int64_t)sigma[i] * ldS;
    uint32_t *dst = Snext + (int64_t)i * ldS;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i; j += gridDim.x * blockDim.x)
        dst[j] = src[sigma[j]];
}

// Append the panel's pivots, D and zero rows (as original indices) to the
// global lists.
__global__ void record_panel_kernel(const PanelOut *__restrict__ out, const int *__restrict__ idx,
                                    int r0, int z0, int *piv_all, uint32_t *d_all,
                                    uint32_t *e_all, int *zero_all, int *zero_cols)
{
    const int np = out->np, nz = out->nzero;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        piv_all[r0 + k] = idx[out->piv_rows[k]];
        d_all[r0 + k] = out->dval[k];
        e_all[r0 + k] = out->eval[k];
    }
    for (int q = threadIdx.x; q < nz; q += blockDim.x) {
        zero_all[z0 + q] = idx[out->zero_rows[q]];
        zero_cols[z0 + q] = r0 + out->zero_np[q];  // L columns that existed when it was found zero
    }
}

// Final output (PERM of Algorithm 2 applied to L): row k of the result is the
// L row of original row perm[k].  Strictly lower part: L (columns >= r are
// identity columns, so zero there; a non-pivot row is zero in every column
// created after it was found zero); diagonal: D_kk.  One CTA per row; with
// 16-byte aligned rows of A (vec) the row moves in 16-byte chunks (Lw rows are
// 256-byte aligned), the chunk that holds the diagonal element by element.
__global__ void __launch_bounds__(256) finalize_kernel(int64_t n, const uint32_t *__restrict__ Lw, int64_t ldw,
                                                       const int *__restrict__ piv_all,
                                                       const uint32_t *__restrict__ d_all,
                                                       const uint32_t *__restrict__ e_all,
                                                       const int *__restrict__ zero_all,
                                                       const int *__restrict__ zero_cols, int r,
                                                       uint32_t *__restrict__ A, int64_t lda,
                                                       int32_t *__restrict__ perm, uint32_t *__restrict__ e,
                                                       int64_t *__restrict__ rank, int vec)
{
    const int64_t k = blockIdx.x;
    if (k >= n) return;
    const int src = (k < r) ? piv_all[k] : zero_all[k - r];
    if (threadIdx.x == 0) {
        perm[k] = src;
        e[k] = (k < r) ? e_all[k] : 0u;
        if (k == 0) *rank = r;
    }
    const uint32_t *lrow = Lw + (int64_t)src * ldw;
    uint32_t *arow = A + k * lda;
    const int64_t cmax = (k < r) ? k : (int64_t)zero_cols[k - r];
    const uint32_t dk = (k < r) ? d_all[k] : 0u;
    int64_t c0 = 0;
    if (vec) {
        const int64_t nfull = k >> 2;  // chunks strictly left of the diagonal
        const uint4 *l4 = reinterpret_cast<const uint4 *>(lrow);
        uint4 *a4 = reinterpret_cast<uint4 *>(arow);
        for (int64_t q = threadIdx.x; q < nfull; q += blockDim.x) {
            const int64_t c = q << 2;
            uint4 v;
            if (c + 3 < cmax) {
                v = __ldg(l4 + q);
            } else {
                v.x = c < cmax ? __ldg(lrow + c) : 0u;
                v.y = c + 1 < cmax ? __ldg(lrow + c + 1) : 0u;
                v.z = c + 2 < cmax ? __ldg(lrow + c + 2) : 0u;
                v.w = 0u;  // c + 3 >= cmax
            }
            a4[q] = v;
        }
        c0 = nfull << 2;
    }
    for (int64_t c = c0 + threadIdx.x; c <= k; c += blockDim.x) {
        uint32_t v;
        if (c == k) v = dk;
        else if (c < cmax) v = __ldg(lrow + c);
        else v = 0u;
        arow[c] = v;
    }
}

__global__ void rpm_clear_kernel(int64_t n, int32_t *rpm_col)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rpm_col[i] = -1;
}

// R_A = P Psi P^T: Psi_kk = 1 for a 1x1 block, Psi = J on a 2x2 block.
__global__ void rpm_kernel(int64_t n, const int32_t *__restrict__ perm, const uint32_t *__restrict__ e,
                           const int64_t *__restrict__ rank, int32_t *__restrict__ rpm_col)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = *rank;
    if (k >= r) return;
    if (e[k] != 0) {
        int a = perm[k], b = perm[k + 1];
        rpm_col[a] = b;
        rpm_col[b] = a;
    } else if (k == 0 || e[k - 1] == 0) {
        int a = perm[k];
        rpm_col[a] = a;
    }
}

inline unsigned gx_for(int64_t len, int threads)
{
    int64_t g = (len + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 64) g = 64;
    return (unsigned)g;
}

}  // namespace

cudaError_t launch_ingest(const uint32_t *A, int64_t lda, int64_t n, uint32_t *S, int64_t ldS,
                          int *idx, FieldP f, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int vec = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
    ingest_kernel<<<(unsigned)n, 256, 0, st>>>(A, lda, n, S, ldS, idx, f, vec);
    return cudaGetLastError();
}

cudaError_t launch_ingest_perm(const uint32_t *A, int64_t lda, int64_t n, const int32_t *perm, uint32_t *S,
                               int64_t ldS, int *idx, FieldP f, int *bad, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    dim3 grid(gx_for(n, 256), (unsigned)n);
    ingest_perm_kernel<<<grid, 256, 0, st>>>(A, lda, n, perm, S, ldS, idx, f, bad);
    return cudaGetLastError();
}

cudaError_t launch_lw_scatter(const uint32_t *LpT, int64_t ldL, int m, int np, const int *idx,
                              uint32_t *Lw, int64_t ldw, int col0, cudaStream_t st)
{
    if (m == 0 || np == 0) return cudaSuccess;
    dim3 grid((m + 31) / 32, (np + 31) / 32);
    lw_scatter_kernel<<<grid, dim3(32, 8), 0, st>>>(LpT, ldL, m, np, idx, Lw, ldw, col0);
    return cudaGetLastError();
}

cudaError_t launch_compact_copy(const uint32_t *S, int64_t ldS, const int *sigma, int m_next,
                                uint32_t *Snext, cudaStream_t st)
{
    if (m_next == 0) return cudaSuccess;
    dim3 grid(gx_for(m_next, 256), (unsigned)m_next);
    compact_copy_kernel<<<grid, 256, 0, st>>>(S, ldS, sigma, m_next, Snext);
    return cudaGetLastError();
}

cudaError_t launch_record_panel(const PanelOut *out, const int *idx, int r0, int z0, int *piv_all,
                                uint32_t *d_all, uint32_t *e_all, int *zero_all, int *zero_cols,
                                cudaStream_t st)
{
    record_panel_kernel<<<1, 256, 0, st>>>(out, idx, r0, z0, piv_all, d_all, e_all, zero_all, zero_cols);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int64_t n, const uint32_t *Lw, int64_t ldw, const int *piv_all,
                            const uint32_t *d_all, const uint32_t *e_all, const int *zero_all,
                            const int *zero_cols, int r, uint32_t *A, int64_t lda, int32_t *perm,
                            uint32_t *e, int64_t *rank, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int vec = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0) && (ldw % 4 == 0);
    finalize_kernel<<<(unsigned)n, 256, 0, st>>>(n, Lw, ldw, piv_all, d_all, e_all, zero_all, zero_cols, r,
                                                 A, lda, perm, e, rank, vec);
    return cudaGetLastError();
}

cudaError_t launch_rpm(int64_t n, const int32_t *perm, const uint32_t *e, const int64_t *rank,
                       int32_t *rpm_col, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    unsigned g = (unsigned)((n + 255) / 256);
    rpm_clear_kernel<<<g, 256, 0, st>>>(n, rpm_col);
    rpm_kernel<<<g, 256, 0, st>>>(n, perm, e, rank, rpm_col);
    return cudaGetLastError();
}
