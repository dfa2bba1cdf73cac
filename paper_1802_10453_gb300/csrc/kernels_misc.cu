// kernels_misc.cu -- the HBM-streaming steps around the pivot chain:
// ingest of A, storing the panel's L columns, the panel loop's state, the
// final symmetric permutation of L
// (PERM of Algorithm 2) and the rank profile matrix P Psi P^T (Section 2.1).
#include "../../include/ldlt_rpm.h"
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

// Lw[idx[t]][r0 + j] = LpC[j][t] for the panel's np columns and m rows:
// transpose through shared memory so both the reads (along t) and the writes
// (along j) are coalesced.
__global__ void lw_scatter_kernel(const uint32_t *__restrict__ LpC, int64_t ldL,
                                  const LoopState *__restrict__ ls, const PanelOut *__restrict__ out,
                                  const int *__restrict__ idx, uint32_t *__restrict__ Lw, int64_t ldw)
{
    if (!step_live(ls, out)) return;
    const int m = ls->m, np = out->np, col0 = ls->r0;
    __shared__ uint32_t tile[32][33];
    const int t0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    if (t0 >= m || j0 >= np) return;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        int j = j0 + r, t = t0 + tx;
        if (j < np && t < m) tile[r][tx] = LpC[(int64_t)j * ldL + t];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        int t = t0 + r, j = j0 + tx;
        if (t < m && j < np) Lw[(int64_t)idx[t] * ldw + col0 + j] = tile[tx][r];
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
                                                       const int *__restrict__ zero_cols,
                                                       const LoopState *__restrict__ ls,
                                                       uint32_t *__restrict__ A, int64_t lda,
                                                       int32_t *__restrict__ perm, uint32_t *__restrict__ e,
                                                       int64_t *__restrict__ rank, int vec)
{
    const int64_t k = blockIdx.x;
    if (k >= n || ls->aborted) return;  // an aborted factorisation leaves the outputs alone
    const int r = ls->r0;
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

// Start (init) or advance the panel loop; see launch_loop_step.  Block 0
// updates the state; every block clears its share of the next panel's
// partner flags, sized from the panel record alone (never from the state
// block 0 is writing).
__global__ void __launch_bounds__(256) loop_step_kernel(LoopState *ls, const PanelOut *out, int init, int64_t n,
                                                        int32_t *status, uint8_t *consumed, PanelSync *sync,
                                                        cudaGraphConditionalHandle cond, int set_cond)
{
    const int mclr = init ? (int)n : (out->abort ? 0 : out->m_next);
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t t = tid; t < mclr; t += nthr) consumed[t] = 0;
    if (blockIdx.x != 0) return;
    if (threadIdx.x == 0) {
        *sync = PanelSync{0, 0, 0, 0};
        if (init) {
            *ls = LoopState{(int)n, 0, 0, 0, 0, 0, {0, 0}};
        } else if (!ls->done) {
            ls->npanel += 1;
            if (out->abort || *(volatile int32_t *)status != 0) {
                ls->done = 1;
                ls->aborted = 1;
            } else if (out->m_next >= ls->m) {
                // a panel always retires a row; this guard keeps the loop finite
                atomicCAS(status, 0, LDLT_ERR_INTERNAL);
                ls->done = 1;
                ls->aborted = 1;
            } else {
                ls->r0 += out->np;
                ls->z0 += out->nzero;
                ls->m = out->m_next;
                if (out->m_next == 0) ls->done = 1;
            }
        }
        if (set_cond) cudaGraphSetConditional(cond, ls->done ? 0u : 1u);
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

cudaError_t launch_lw_scatter(const uint32_t *LpC, int64_t ldL, int64_t n, const LoopState *ls,
                              const PanelOut *out, const int *idx, uint32_t *Lw, int64_t ldw,
                              cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 31) / 32), KP_MAX / 32);
    lw_scatter_kernel<<<grid, dim3(32, 8), 0, st>>>(LpC, ldL, ls, out, idx, Lw, ldw);
    return cudaGetLastError();
}

cudaError_t launch_loop_step(LoopState *ls, const PanelOut *out, int init, int64_t n, int32_t *status,
                             uint8_t *consumed, PanelSync *sync, cudaGraphConditionalHandle cond, int set_cond,
                             int num_sms, cudaStream_t st)
{
    int64_t g = (n + 255) / 256;
    if (g > 2 * num_sms) g = 2 * num_sms;
    if (g < 1) g = 1;
    loop_step_kernel<<<(unsigned)g, 256, 0, st>>>(ls, out, init, n, status, consumed, sync, cond, set_cond);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int64_t n, const uint32_t *Lw, int64_t ldw, const int *piv_all,
                            const uint32_t *d_all, const uint32_t *e_all, const int *zero_all,
                            const int *zero_cols, const LoopState *ls, uint32_t *A, int64_t lda,
                            int32_t *perm, uint32_t *e, int64_t *rank, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int vec = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0) && (ldw % 4 == 0);
    finalize_kernel<<<(unsigned)n, 256, 0, st>>>(n, Lw, ldw, piv_all, d_all, e_all, zero_all, zero_cols, ls,
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
