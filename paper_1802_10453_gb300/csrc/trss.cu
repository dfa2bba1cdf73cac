// trss.cu -- Algorithm 1 (TRSS, Problem 1): the upper triangular X with
// X^T U + U^T X = C over Z/pZ, for U upper triangular with a non-zero
// diagonal and C symmetric.  X overwrites C's upper triangle in place (the
// remark after Algorithm 1).
//
// Algorithm 1 halves recursively: X1 from (U1, C1); D2 = C2 - X1^T U2 (TRMM);
// X2 = U1^{-T} D2 (TRSM); D3 = C3 - (X2^T U2 + U2^T X2) (SYR2K); X3 from
// (U3, D3).  Unrolled over blocks of TB rows from the top it is the
// right-looking form, run here in two forms (block k = rows [k0, k1)).
// ldlt_rpm_trss (CUDA cores), three launches per block:
//   trss_diag_kernel   X_kk from U_kk and C_kk: the same steps with blocks of
//                      one row, in one CTA (x_ii = c_ii / (2 u_ii), the row
//                      to its right, a rank-2 update of the rest of the block)
//   trss_panel_kernel  X_k,r = U_kk^{-T} (C_k,r - X_kk^T U_k,r) for the
//                      columns r >= k1, a warp per column
//   trss_syr2k_kernel  C_r,r -= X_k,r^T U_k,r + U_k,r^T X_k,r on the upper
//                      triangle of the trailing block, 64 x 64 tiles
// ldlt_rpm_trss_ws (tensor cores), blocks of TW = 64 rows: the inverses
// V_k = U_kk^{-1} of all diagonal blocks once (trss_vinv_kernel), then two
// launches per block:
//   trss_step_kernel   X_kk by dense products with V_k (no substitution
//                      chain), the panel X_k,r = V_k^T (C_k,r - X_kk^T U_k,r),
//                      and the trailing update's limb operands
//   syrdk_tc_kernel    the SYR2K on tcgen05 (upper-triangle mode) for
//                      trailing orders >= 256; trss_syr2k_kernel below
// Characteristic 2: the diagonal of X^T U + U^T X is zero, so a solution
// exists only if C's diagonal (after the updates) is zero; x_ii = 0 is taken
// and a non-zero diagonal entry is reported as LDLT_ERR_INCONSISTENT.
// Arithmetic: residues < p < 2^31, exact 64-bit products; sums are folded
// below 2^63 by subtracting a multiple of p (field.cuh), reduced once.
#include <cstdint>

#include "../../include/ldlt_rpm.h"
#include "ldlt_internal.cuh"
#include "tc_split.cuh"

namespace {

constexpr int TB = 32;      // rows per block step
constexpr int TC = 64;      // columns per CTA tile of the trailing kernel

__device__ __forceinline__ uint32_t rd(const uint32_t *M, int64_t ld, int64_t i, int64_t j, const FieldP &f)
{
    const uint32_t v = M[i * ld + j];
    return v >= f.p ? v % f.p : v;
}

// X_kk: TB x TB (nb x nb used) in one CTA of TB * TB threads.  Thread (r, l)
// (warp r, lane l) owns c_rl (r <= l) and the sum of the rank-2 terms it has
// received.  Step i: warp i finishes row i of X (lane i forms x_ii, a shuffle
// broadcasts it, x_il = (c_il - x_ii u_il) / u_ii) and stores it; after one
// barrier every later row r adds x_ir u_il + u_ir x_il to its sum, which is
// reduced only when its row comes.  For p < 2^28 the sums of at most 2 TB
// products (each < 2^56) stay below 2^63; larger p fold after every product.
template <bool BIG>
__global__ void __launch_bounds__(TB * TB) trss_diag_kernel(int64_t k0, int nb, const uint32_t *U, int64_t ldu,
                                                            uint32_t *C, int64_t ldc, int32_t *status, FieldP f)
{
    __shared__ uint32_t u[TB][TB + 1], x[TB][TB + 1], uinv[TB];
    const int l = threadIdx.x % TB, r = threadIdx.x / TB;
    const bool in = r < nb && l < nb && r <= l;
    u[r][l] = in ? rd(U, ldu, k0 + r, k0 + l, f) : 0u;
    const uint32_t crl = in ? rd(C, ldc, k0 + r, k0 + l, f) : 0u;
    x[r][l] = 0u;
    __syncthreads();
    if (threadIdx.x < nb) {
        const uint32_t d = u[threadIdx.x][threadIdx.x];
        if (d == 0u) {
            atomicExch(status, LDLT_ERR_ARG);
            uinv[threadIdx.x] = 0u;
        } else {
            uinv[threadIdx.x] = fp_inv(d, f);
        }
    }
    __syncthreads();
    uint64_t acc = 0;
    for (int i = 0; i < nb; ++i) {
        if (r == i) {
            const uint32_t ci = fp_sub(crl, fp_reduce64(acc, f), f);  // c_il after steps < i
            uint32_t xii = 0;
            if (l == i) {
                if (f.p == 2u) {
                    if (ci != 0u) atomicExch(status, LDLT_ERR_INCONSISTENT);
                } else {
                    xii = fp_mul(fp_mul(ci, f.inv2, f), uinv[i], f);
                }
            }
            xii = __shfl_sync(0xffffffffu, xii, i);
            uint32_t xil = 0;
            if (l == i) xil = xii;
            else if (l > i && l < nb) xil = fp_mul(fp_sub(ci, fp_mul(xii, u[i][l], f), f), uinv[i], f);
            x[i][l] = xil;
        }
        __syncthreads();
        if (r > i && r <= l && l < nb) {
            if (BIG) {
                fp_mac(acc, x[i][r], u[i][l], f);
                fp_mac(acc, u[i][r], x[i][l], f);
            } else {
                acc += (uint64_t)x[i][r] * u[i][l] + (uint64_t)u[i][r] * x[i][l];
            }
        }
    }
    if (in) C[(k0 + r) * ldc + k0 + l] = x[r][l];
}

// X_k,r for the columns r >= k1 of the trailing part, one warp per column j
// and one lane per row i of the block: t_i = C_ij - sum_{k <= i} X_ki U_kj
// (the column of U held one entry per lane and broadcast by shuffles), then
// U_kk^T y = t right-looking: lane i finishes y_i, it is broadcast, and the
// lanes below add u_il y_i.  Each of the nb steps of the substitution costs
// one reduction, one product and one shuffle on the dependent chain, and all
// columns of the step run side by side.  For p < 2^28 a lane's sum of at most
// 2 TB products (each < 2^56) stays below 2^63 without folding.
constexpr int PW = 8;  // columns (warps) per CTA in the panel kernel
template <bool BIG>
__global__ void __launch_bounds__(PW * 32) trss_panel_kernel(int64_t k0, int nb, int64_t n, const uint32_t *U,
                                                              int64_t ldu, uint32_t *C, int64_t ldc, FieldP f)
{
    __shared__ uint32_t u[TB][TB + 1], x[TB][TB + 1], uinv[TB];
    const int64_t k1 = k0 + nb;
    for (int q = threadIdx.x; q < TB * TB; q += blockDim.x) {
        const int r = q / TB, s = q % TB;
        const bool in = r < nb && s < nb && r <= s;
        u[r][s] = in ? rd(U, ldu, k0 + r, k0 + s, f) : 0u;
        x[r][s] = in ? C[(k0 + r) * ldc + k0 + s] : 0u;  // X_kk, already reduced
    }
    __syncthreads();
    if (threadIdx.x < nb) {
        const uint32_t d = u[threadIdx.x][threadIdx.x];
        uinv[threadIdx.x] = d ? fp_inv(d, f) : 0u;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = k1 + (int64_t)blockIdx.x * PW + warp;
    if (j >= n) return;  // whole warps
    const bool row = lane < nb;
    const uint32_t ucj = row ? rd(U, ldu, k0 + lane, j, f) : 0u;
    const uint32_t ccj = row ? rd(C, ldc, k0 + lane, j, f) : 0u;
    uint64_t acc = 0;
    for (int k = 0; k < nb; ++k) {  // acc_i = sum_{k <= i} x_ki u_kj (x is upper triangular)
        const uint32_t ukj = __shfl_sync(0xffffffffu, ucj, k);
        if (BIG) fp_mac(acc, x[k][lane], ukj, f);
        else acc += (uint64_t)x[k][lane] * ukj;
    }
    uint32_t y = 0;
    for (int i = 0; i < nb; ++i) {
        uint32_t yi = 0;
        if (lane == i) {
            yi = fp_mul(fp_sub(ccj, fp_reduce64(acc, f), f), uinv[i], f);
            y = yi;
        }
        yi = __shfl_sync(0xffffffffu, yi, i);
        if (lane > i) {
            if (BIG) fp_mac(acc, u[i][lane], yi, f);
            else acc += (uint64_t)u[i][lane] * yi;
        }
    }
    if (row) C[(k0 + lane) * ldc + j] = y;
}

// C[i][j] -= sum_k (X[k][i] U[k][j] + U[k][i] X[k][j]) for the nb <= TB rows
// k of block rows k0 .. k0+nb-1, k1 <= i <= j < n (k1 >= k0 + nb: the first
// trailing index, which a 64-row block updates in two 32-row halves); one
// 64 x 64 tile per CTA, 4 x 4 outputs per thread.  For p < 2^28 the 2 TB
// products (each < 2^56) sum below 2^63 without folding; larger p fold after
// every product.
template <bool BIG>
__global__ void __launch_bounds__(256) trss_syr2k_kernel(int64_t k0, int nb, int64_t k1, int64_t n,
                                                          const uint32_t *U, int64_t ldu, uint32_t *C, int64_t ldc,
                                                          FieldP f)
{
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bi > bj) return;  // tiles wholly below the diagonal
    const int64_t i0 = k1 + (int64_t)bi * TC, j0 = k1 + (int64_t)bj * TC;
    __shared__ uint32_t xi[TB][TC], ui[TB][TC], xj[TB][TC], uj[TB][TC];
    for (int q = threadIdx.x; q < TB * TC; q += blockDim.x) {
        const int k = q / TC, c = q % TC;
        const bool ki = k < nb;
        const int64_t ci = i0 + c, cj = j0 + c;
        xi[k][c] = (ki && ci < n) ? C[(k0 + k) * ldc + ci] : 0u;
        ui[k][c] = (ki && ci < n) ? rd(U, ldu, k0 + k, ci, f) : 0u;
        xj[k][c] = (ki && cj < n) ? C[(k0 + k) * ldc + cj] : 0u;
        uj[k][c] = (ki && cj < n) ? rd(U, ldu, k0 + k, cj, f) : 0u;
    }
    __syncthreads();
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;  // rows ty + 16a, columns tx + 16b
    uint64_t acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    for (int k = 0; k < nb; ++k) {
        uint32_t xa[4], ua[4], xb[4], ub[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            xa[a] = xi[k][ty + 16 * a];
            ua[a] = ui[k][ty + 16 * a];
            xb[a] = xj[k][tx + 16 * a];
            ub[a] = uj[k][tx + 16 * a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (BIG) {
                    fp_mac(acc[a][b], xa[a], ub[b], f);
                    fp_mac(acc[a][b], ua[a], xb[b], f);
                } else {
                    acc[a][b] += (uint64_t)xa[a] * ub[b] + (uint64_t)ua[a] * xb[b];
                }
            }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
            if (i < n && j < n && i <= j) {
                uint32_t *cp = C + i * ldc + j;
                const uint32_t old = *cp >= f.p ? *cp % f.p : *cp;
                *cp = fp_sub(old, fp_reduce64(acc[a][b], f), f);
            }
        }
}

// 64-bit sum of products a b of residues: exact for p < 2^28 over up to 64
// products (each < 2^56); larger p fold after every product.
template <bool BIG>
__device__ __forceinline__ void mac2(uint64_t &acc, uint32_t a, uint32_t b, const FieldP &f)
{
    if (BIG) fp_mac(acc, a, b, f);
    else acc += (uint64_t)a * (uint64_t)b;
}

// V_k = U_kk^{-1} for every TW-row diagonal block of U (upper triangular,
// TW x TW, row-major at V + k TW^2), once per call: U is not changed by the
// solve.  One warp per block, lane i computes rows i and i + 32 of V from
// V U = I:
//   v_ii = 1 / u_ii,   v_il = -(sum_{i <= k < l} v_ik u_kl) / u_ll  (l > i).
// A zero diagonal entry of U is reported as LDLT_ERR_ARG.  For p < 2^28 the
// sums of at most TW - 1 products (each < 2^56) stay below 2^62.
constexpr int TW = 64;  // rows per block step of the tensor-core form
constexpr int TWP = TW + 1;
template <bool BIG>
__global__ void __launch_bounds__(32) trss_vinv_kernel(const uint32_t *U, int64_t ldu, int64_t n, uint32_t *V,
                                                      int32_t *status, FieldP f)
{
    __shared__ uint32_t u[TW][TWP], v[TW][TWP];
    const int lane = threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.x * TW;
    const int nb = (int)(n - k0 < TW ? n - k0 : TW);
    for (int r = 0; r < TW; ++r)
        for (int c = lane; c < TW; c += 32) {
            u[r][c] = (r < nb && c < nb && r <= c) ? rd(U, ldu, k0 + r, k0 + c, f) : 0u;
            v[r][c] = 0u;
        }
    __syncwarp();
    uint32_t ui[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        const uint32_t d = i < nb ? u[i][i] : 1u;
        if (d == 0u) atomicCAS(status, 0, LDLT_ERR_ARG);
        ui[h] = d ? fp_inv(d, f) : 0u;
        if (i < nb) v[i][i] = ui[h];
    }
    for (int l = 1; l < nb; ++l) {
        const uint32_t ul = __shfl_sync(0xffffffffu, l < 32 ? ui[0] : ui[1], l & 31);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = lane + 32 * h;
            if (i < l) {
                uint64_t acc = 0;
                for (int k = i; k < l; ++k) mac2<BIG>(acc, v[i][k], u[k][l], f);
                const uint32_t sl = fp_reduce64_fold(acc, f);
                v[i][l] = fp_mul(sl ? f.p - sl : 0u, ul, f);
            }
        }
    }
    __syncwarp();
    uint32_t *Vk = V + (int64_t)blockIdx.x * TW * TW;
    for (int r = 0; r < TW; ++r)
        for (int c = lane; c < TW; c += 32) Vk[r * TW + c] = v[r][c];
}

// One block step of the tensor-core form in one launch (block k = TW rows
// from k0).  With V = U_kk^{-1} (precomputed) the diagonal problem
// X^T U + U^T X = C_kk is solved without a sequential substitution: M = X V
// is upper triangular and M + M^T = V^T C_kk V =: S, so M takes S's strict
// upper triangle and half its diagonal (characteristic 2: a zero diagonal,
// and S_ii != 0 means the system has no solution) and X_kk = M U_kk -- three
// dense TW x TW products.  Each of the CTA's 32 warps then solves one column
// j >= k1 of the panel, X_k,j = V^T (C_k,j - X_kk^T U_k,j) (two products by
// triangular matrices, a lane per two block rows), and (SPLIT) the CTA writes
// its 32 rows i = j - k1 of the trailing update's limb operands,
// G[i] = [X_k,i | U_k,i] and GD[i] = [U_k,i | X_k,i], so that
// GD G^T = U^T X + X^T U (K = 2 TW = 128; rows past the last column are the
// zero rows that pad the operands to 128).  The solution is unique (for
// p = 2 once x_ii = 0), so it equals the one Algorithm 1's recursion
// computes, bit for bit.  C_kk is read by every CTA, so X_kk is not written
// back here: CTA 0 keeps it in xcur and the next step's CTA 0 (which does not
// read block k) stores it into C; a launch with no trailing columns (the last
// block, one CTA) stores its own.  Thread t computes the outputs (t / 16,
// t mod 16 + 16 q), q < 4, of each TW x TW product.
struct TrssStep {
    int64_t k0, n, ldu, ldc;
    int nb;
    const uint32_t *U;
    const uint32_t *V;      // U_kk^{-1} of every diagonal block
    uint32_t *C;
    int32_t *status;
    FieldP f;
    const uint32_t *xprev;  // X of the previous block (TW x TW, row-major), or null
    int64_t kprev;
    int nbprev;
    uint32_t *xcur;         // this block's X for the next step
    SplitArgs sa;           // SPLIT: operand buffers and digit bases
    PanelOut *out;          // SPLIT: the update record the SYRDK kernel reads
};

constexpr int STEP_THREADS = 1024;
constexpr size_t STEP_SMEM = (size_t)(4 * TW * TWP + 2 * 32 * TWP) * 4;  // u, V, C/M, T1/X; ys, us

template <bool BIG, bool SPLIT>
__global__ void __launch_bounds__(STEP_THREADS) trss_step_kernel(const TrssStep s)
{
    extern __shared__ uint32_t sm[];
    uint32_t(*u)[TWP] = reinterpret_cast<uint32_t(*)[TWP]>(sm);
    uint32_t(*vv)[TWP] = u + TW;
    uint32_t(*c)[TWP] = vv + TW;   // C_kk, then M
    uint32_t(*t1)[TWP] = c + TW;   // C_kk V, then X_kk
    uint32_t(*ys)[TWP] = t1 + TW;  // 32 rows: X_k,j of the CTA's columns
    uint32_t(*us)[TWP] = ys + 32;  // 32 rows: U_k,j
    const FieldP f = s.f;
    const int nb = s.nb;
    const int64_t k0 = s.k0, k1 = k0 + nb, rest = s.n - k1;
    const int tid = threadIdx.x;
    const int r = tid >> 4, l0 = tid & 15;  // outputs (r, l0 + 16 q)
    if (blockIdx.x == 0 && s.xprev)
        for (int q = 0; q < 4; ++q) {
            const int l = l0 + 16 * q;
            if (r < s.nbprev && l < s.nbprev && r <= l)
                s.C[(s.kprev + r) * s.ldc + s.kprev + l] = s.xprev[r * TW + l];
        }
    for (int q = 0; q < 4; ++q) {
        const int l = l0 + 16 * q;
        const bool sq = r < nb && l < nb;
        u[r][l] = (sq && r <= l) ? rd(s.U, s.ldu, k0 + r, k0 + l, f) : 0u;
        vv[r][l] = s.V[(k0 / TW) * TW * TW + r * TW + l];  // zero outside the upper nb x nb triangle
        c[r][l] = sq ? rd(s.C, s.ldc, k0 + (r < l ? r : l), k0 + (r < l ? l : r), f) : 0u;  // symmetric
    }
    __syncthreads();
    // ---- X_kk: T1 = C V, S = V^T T1, M from S, X = M U ----
    {
        uint64_t acc[4] = {0, 0, 0, 0};
        for (int k = 0; k < TW; ++k) {
            const uint32_t crk = c[r][k];
#pragma unroll
            for (int q = 0; q < 4; ++q) mac2<BIG>(acc[q], crk, vv[k][l0 + 16 * q], f);  // V upper: 0 for k > l
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) t1[r][l0 + 16 * q] = fp_reduce64_fold(acc[q], f);
    }
    __syncthreads();
    uint32_t mrl[4];
    {
        uint64_t acc[4] = {0, 0, 0, 0};
        for (int k = 0; k <= r; ++k) {
            const uint32_t vkr = vv[k][r];
#pragma unroll
            for (int q = 0; q < 4; ++q) mac2<BIG>(acc[q], vkr, t1[k][l0 + 16 * q], f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = l0 + 16 * q;
            const uint32_t srl = fp_reduce64_fold(acc[q], f);
            mrl[q] = 0u;
            if (r < l) mrl[q] = srl;
            else if (r == l) {
                if (f.p != 2u) mrl[q] = fp_mul(srl, f.inv2, f);
                else if (srl != 0u && r < nb && blockIdx.x == 0) atomicCAS(s.status, 0, LDLT_ERR_INCONSISTENT);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) c[r][l0 + 16 * q] = mrl[q];  // M (C_kk is no longer needed)
    __syncthreads();
    {
        uint64_t acc[4] = {0, 0, 0, 0};
        for (int k = r; k < TW; ++k) {
            const uint32_t mrk = c[r][k];
#pragma unroll
            for (int q = 0; q < 4; ++q) mac2<BIG>(acc[q], mrk, u[k][l0 + 16 * q], f);  // U upper: 0 for k > l
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) t1[r][l0 + 16 * q] = fp_reduce64_fold(acc[q], f);  // X_kk
    }
    __syncthreads();
    uint32_t(*x)[TWP] = t1;
    if (blockIdx.x == 0)
        for (int q = 0; q < 4; ++q) {
            const int l = l0 + 16 * q;
            if (r < nb && l < nb && r <= l) {
                if (rest > 0) s.xcur[r * TW + l] = x[r][l];
                else s.C[(k0 + r) * s.ldc + k0 + l] = x[r][l];
            }
        }
    // ---- panel column j (warp w, lane: block rows lane and lane + 32) ----
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t i = (int64_t)blockIdx.x * 32 + warp;  // trailing index
    const int64_t j = k1 + i;
    uint32_t y[2] = {0u, 0u}, ucj[2] = {0u, 0u};
    if (i < rest) {
        uint32_t ccj[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int b = lane + 32 * h;
            ucj[h] = b < nb ? rd(s.U, s.ldu, k0 + b, j, f) : 0u;
            ccj[h] = b < nb ? rd(s.C, s.ldc, k0 + b, j, f) : 0u;
        }
        uint64_t a0 = 0, a1 = 0;
        for (int k = 0; k < nb; ++k) {  // sum_{k <= b} x_kb u_kj (x is upper triangular)
            const uint32_t ukj = __shfl_sync(0xffffffffu, k < 32 ? ucj[0] : ucj[1], k & 31);
            mac2<BIG>(a0, x[k][lane], ukj, f);
            mac2<BIG>(a1, x[k][lane + 32], ukj, f);
        }
        const uint32_t t0 = fp_sub(ccj[0], fp_reduce64_fold(a0, f), f);
        const uint32_t t1v = fp_sub(ccj[1], fp_reduce64_fold(a1, f), f);
        a0 = 0; a1 = 0;
        for (int k = 0; k < nb; ++k) {  // y = V^T t
            const uint32_t tk = __shfl_sync(0xffffffffu, k < 32 ? t0 : t1v, k & 31);
            mac2<BIG>(a0, vv[k][lane], tk, f);
            mac2<BIG>(a1, vv[k][lane + 32], tk, f);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int b = lane + 32 * h;
            y[h] = b < nb ? fp_reduce64_fold(h ? a1 : a0, f) : 0u;
            if (b < nb) s.C[(k0 + b) * s.ldc + j] = y[h];
        }
    }
    if (SPLIT) {
        const int np = 2 * nb, kpad = (np + 63) / 64 * 64;
        const int rows = (int)((rest + TC_BM - 1) / TC_BM * TC_BM), kprime = s.sa.la * kpad;
        if (blockIdx.x == 0 && tid == 0) {
            s.out->m_next = (int)rest;
            s.out->np = np;
            s.out->abort = 0;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            ys[warp][lane + 32 * h] = y[h];
            us[warp][lane + 32 * h] = ucj[h];
        }
        __syncthreads();
        // thread t < 32 * kpad / 8 forms columns 8g .. 8g+7 (g = t mod kpad/8) of
        // the CTA's row t / (kpad/8): G = [X | U], GD = [U | X]
        const int ng = kpad / 8;
        const int w = tid / ng, g = tid % ng;
        const int64_t iw = (int64_t)blockIdx.x * 32 + w;
        if (w < 32 && iw < rows) {
            int32_t gd_bal[8];
            uint32_t gk[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = 8 * g + e;
                gk[e] = k < nb ? ys[w][k] : (k < np ? us[w][k - nb] : 0u);
                gd_bal[e] = balanced(k < nb ? us[w][k] : (k < np ? ys[w][k - nb] : 0u), f.p);
            }
            split_write(s.sa, (int)iw, 8 * g, kpad, kprime, rows, gd_bal, gk);
        }
    }
}

__global__ void trss_iota_kernel(int *sigma, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        sigma[i] = (int)i;
}

constexpr int TRSS_TC_MIN = 256;  // trailing orders below this keep the CUDA-core SYR2K

// Workspace of the tensor-core form: loop state and update record (read by
// the SYRDK kernel), the identity row map, the limb operands.
struct TrssLayout {
    size_t ls, out, sigma, uinv, xblk, opA, opB, total;
};

void trss_layout(int64_t n, uint32_t p, TrssLayout &L)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const int limbs = tc_limbs(p);
    L.ls = take(sizeof(LoopState));
    L.out = take(sizeof(PanelOut));
    L.sigma = take((size_t)(n > 0 ? n : 1) * 4);
    const int64_t nn = n > 0 ? n : 1;
    L.uinv = take((size_t)round_up(nn, TW) * TW * 4);  // U_kk^{-1} of every diagonal block
    L.xblk = take((size_t)2 * TW * TW * 4);
    L.opA = take(tc_operand_bytes(nn, limbs));
    L.opB = L.opA + (size_t)round_up(round_up(nn, 128) * (int64_t)limbs * KP_MAX * 2, 256);
    L.total = off;
}

}  // namespace

extern "C" int ldlt_rpm_trss_workspace_bytes(int64_t n, uint32_t p, size_t *bytes)
{
    size_t tmp = 0;
    const int rc = ldlt_rpm_workspace_bytes(1, p, LDLT_PATH_TC, &tmp);  // p prime, in range
    if (rc != LDLT_OK) return rc;
    if (n < 0 || !bytes) return LDLT_ERR_ARG;
    TrssLayout L;
    trss_layout(n, p, L);
    *bytes = L.total;
    return LDLT_OK;
}

extern "C" int ldlt_rpm_trss_ws(int64_t n, uint32_t p, const uint32_t *U, int64_t ldu, uint32_t *C, int64_t ldc,
                                int32_t *status, void *ws, size_t ws_bytes, void *stream)
{
    size_t need = 0;
    const int rc = ldlt_rpm_trss_workspace_bytes(n, p, &need);
    if (rc != LDLT_OK) return rc;
    if (!status) return LDLT_ERR_ARG;
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255) != 0) return LDLT_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return LDLT_ERR_CUDA;
    if (n == 0) return LDLT_OK;
    if (!U || !C || ldu < n || ldc < n) return LDLT_ERR_ARG;
    int dev = 0, nsm = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return LDLT_ERR_CUDA;
    if (major != 10 || minor != 3) return LDLT_ERR_NO_DEVICE;
    TrssLayout Lo;
    trss_layout(n, p, Lo);
    uint8_t *w = (uint8_t *)ws;
    LoopState *ls = (LoopState *)(w + Lo.ls);
    PanelOut *out = (PanelOut *)(w + Lo.out);
    int *sigma = (int *)(w + Lo.sigma);
    void *opA = w + Lo.opA, *opB = w + Lo.opB;
    const FieldP f = make_field(p);
    const int limbs = tc_limbs(p);
    // loop state "running" and an update record with no abort: the SYRDK kernel's liveness test
    if (cudaMemsetAsync(w, 0, Lo.sigma, st) != cudaSuccess) return LDLT_ERR_CUDA;
    trss_iota_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(sigma, n);
    uint32_t *V = (uint32_t *)(w + Lo.uinv);
    uint32_t *xblk = (uint32_t *)(w + Lo.xblk);
    const bool big = p >= (1u << 28);
    const unsigned nblk = (unsigned)((n + TW - 1) / TW);
    if (big) trss_vinv_kernel<true><<<nblk, 32, 0, st>>>(U, ldu, n, V, status, f);
    else trss_vinv_kernel<false><<<nblk, 32, 0, st>>>(U, ldu, n, V, status, f);
    if (cudaFuncSetAttribute(trss_step_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)STEP_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(trss_step_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)STEP_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(trss_step_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)STEP_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(trss_step_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)STEP_SMEM) != cudaSuccess)
        return LDLT_ERR_CUDA;
    TrssStep sp;
    sp.n = n; sp.ldu = ldu; sp.ldc = ldc; sp.U = U; sp.V = V; sp.C = C; sp.status = status; sp.f = f;
    sp.sa = tc_split_args(f, limbs, opA, opB);
    sp.out = out;
    sp.xprev = nullptr; sp.kprev = 0; sp.nbprev = 0;
    for (int64_t k0 = 0, step = 0; k0 < n; k0 += TW, ++step) {
        const int nb = (int)((n - k0) < TW ? (n - k0) : TW);
        const int64_t k1 = k0 + nb, rest = n - k1;
        const bool tc = rest >= TRSS_TC_MIN;
        sp.k0 = k0; sp.nb = nb;
        sp.xcur = xblk + (step & 1) * TW * TW;
        // one CTA per 32 trailing columns (tensor form: per 32 operand rows, padded to 128)
        const int64_t cols = tc ? round_up(rest, 128) : rest;
        const unsigned grid = (unsigned)(cols > 0 ? (cols + 31) / 32 : 1);
        if (tc) {
            if (big) trss_step_kernel<true, true><<<grid, STEP_THREADS, STEP_SMEM, st>>>(sp);
            else trss_step_kernel<false, true><<<grid, STEP_THREADS, STEP_SMEM, st>>>(sp);
        } else {
            if (big) trss_step_kernel<true, false><<<grid, STEP_THREADS, STEP_SMEM, st>>>(sp);
            else trss_step_kernel<false, false><<<grid, STEP_THREADS, STEP_SMEM, st>>>(sp);
        }
        sp.xprev = sp.xcur; sp.kprev = k0; sp.nbprev = nb;
        if (rest <= 0) continue;
        if (tc) {
            // C_rr -= X^T U + U^T X on tensor cores: the SYRDK kernel on C's upper triangle (K = 2 nb)
            uint32_t *blk = C + k1 * ldc + k1;
            if (launch_syrdk_tc(blk, ldc, sigma, ls, out, opA, opB, limbs, f, blk, 2000000000LL, status, nsm, 0,
                                st, 1) != cudaSuccess)
                return LDLT_ERR_CUDA;
        } else {
            // CUDA cores, the block's rows in halves of TB (the tile kernel holds TB rows)
            const unsigned gp = (unsigned)((rest + TC - 1) / TC);
            for (int h = 0; h < nb; h += TB) {
                const int nh = nb - h < TB ? nb - h : TB;
                if (big) trss_syr2k_kernel<true><<<dim3(gp, gp), 256, 0, st>>>(k0 + h, nh, k1, n, U, ldu, C, ldc, f);
                else trss_syr2k_kernel<false><<<dim3(gp, gp), 256, 0, st>>>(k0 + h, nh, k1, n, U, ldu, C, ldc, f);
            }
        }
    }
    return cudaGetLastError() == cudaSuccess ? LDLT_OK : LDLT_ERR_CUDA;
}

extern "C" int ldlt_rpm_trss(int64_t n, uint32_t p, const uint32_t *U, int64_t ldu, uint32_t *C, int64_t ldc,
                             int32_t *status, void *stream)
{
    size_t tmp = 0;
    const int rc = ldlt_rpm_workspace_bytes(1, p, LDLT_PATH_TC, &tmp);  // p prime, in range
    if (rc != LDLT_OK) return rc;
    if (n < 0 || !status) return LDLT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return LDLT_ERR_CUDA;
    if (n == 0) return LDLT_OK;
    if (!U || !C || ldu < n || ldc < n) return LDLT_ERR_ARG;
    const FieldP f = make_field(p);
    for (int64_t k0 = 0; k0 < n; k0 += TB) {
        const int nb = (int)((n - k0) < TB ? (n - k0) : TB);
        if (p >= (1u << 28)) trss_diag_kernel<true><<<1, TB * TB, 0, st>>>(k0, nb, U, ldu, C, ldc, status, f);
        else trss_diag_kernel<false><<<1, TB * TB, 0, st>>>(k0, nb, U, ldu, C, ldc, status, f);
        const int64_t rest = n - (k0 + nb);
        if (rest <= 0) continue;
        const unsigned gp = (unsigned)((rest + TC - 1) / TC);
        const unsigned gw = (unsigned)((rest + PW - 1) / PW);
        if (p >= (1u << 28))
            trss_panel_kernel<true><<<gw, PW * 32, 0, st>>>(k0, nb, n, U, ldu, C, ldc, f);
        else
            trss_panel_kernel<false><<<gw, PW * 32, 0, st>>>(k0, nb, n, U, ldu, C, ldc, f);
        if (p >= (1u << 28))
            trss_syr2k_kernel<true><<<dim3(gp, gp), 256, 0, st>>>(k0, nb, k0 + nb, n, U, ldu, C, ldc, f);
        else
            trss_syr2k_kernel<false><<<dim3(gp, gp), 256, 0, st>>>(k0, nb, k0 + nb, n, U, ldu, C, ldc, f);
    }
    return cudaGetLastError() == cudaSuccess ? LDLT_OK : LDLT_ERR_CUDA;
}
