// trss.cu -- Algorithm 1 (TRSS, Problem 1): the upper triangular X with
// X^T U + U^T X = C over Z/pZ, for U upper triangular with a non-zero
// diagonal and C symmetric.  X overwrites C's upper triangle in place (the
// remark after Algorithm 1).
//
// Algorithm 1 halves recursively: X1 from (U1, C1); D2 = C2 - X1^T U2 (TRMM);
// X2 = U1^{-T} D2 (TRSM); D3 = C3 - (X2^T U2 + U2^T X2) (SYR2K); X3 from
// (U3, D3).  Unrolled over blocks of TB rows from the top it is the
// right-looking form run here, three launches per block k (rows [k0, k1)):
//   trss_diag_kernel   X_kk from U_kk and C_kk: the same steps with blocks of
//                      one row, in one CTA (x_ii = c_ii / (2 u_ii), the row
//                      to its right, a rank-2 update of the rest of the block)
//   trss_panel_kernel  X_k,r = U_kk^{-T} (C_k,r - X_kk^T U_k,r) for the
//                      columns r >= k1, a warp per column
//   trss_syr2k_kernel  C_r,r -= X_k,r^T U_k,r + U_k,r^T X_k,r on the upper
//                      triangle of the trailing block, 64 x 64 tiles
// Characteristic 2: the diagonal of X^T U + U^T X is zero, so a solution
// exists only if C's diagonal (after the updates) is zero; x_ii = 0 is taken
// and a non-zero diagonal entry is reported as LDLT_ERR_INCONSISTENT.
// Arithmetic: residues < p < 2^31, exact 64-bit products; sums are folded
// below 2^63 by subtracting a multiple of p (field.cuh), reduced once.
#include <cstdint>

#include "../../include/ldlt_rpm.h"
#include "ldlt_internal.cuh"

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

// C[i][j] -= sum_k (X[k][i] U[k][j] + U[k][i] X[k][j]) for k in the block,
// k1 <= i <= j < n; one 64 x 64 tile per CTA, 4 x 4 outputs per thread.  For
// p < 2^28 the 2 TB products of a block (each < 2^56) sum below 2^63 without
// folding; larger p fold after every product.
template <bool BIG>
__global__ void __launch_bounds__(256) trss_syr2k_kernel(int64_t k0, int nb, int64_t n, const uint32_t *U,
                                                          int64_t ldu, uint32_t *C, int64_t ldc, FieldP f)
{
    const int64_t k1 = k0 + nb;
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

__global__ void trss_iota_kernel(int *sigma, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        sigma[i] = (int)i;
}

constexpr int TRSS_TC_MIN = 256;  // trailing orders below this keep the CUDA-core SYR2K

// Workspace of the tensor-core form: loop state and update record (read by
// the SYRDK kernel), the identity row map, the limb operands.
struct TrssLayout {
    size_t ls, out, sigma, opA, opB, total;
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
    for (int64_t k0 = 0; k0 < n; k0 += TB) {
        const int nb = (int)((n - k0) < TB ? (n - k0) : TB);
        if (p >= (1u << 28)) trss_diag_kernel<true><<<1, TB * TB, 0, st>>>(k0, nb, U, ldu, C, ldc, status, f);
        else trss_diag_kernel<false><<<1, TB * TB, 0, st>>>(k0, nb, U, ldu, C, ldc, status, f);
        const int64_t k1 = k0 + nb, rest = n - k1;
        if (rest <= 0) continue;
        const unsigned gw = (unsigned)((rest + PW - 1) / PW);
        if (p >= (1u << 28))
            trss_panel_kernel<true><<<gw, PW * 32, 0, st>>>(k0, nb, n, U, ldu, C, ldc, f);
        else
            trss_panel_kernel<false><<<gw, PW * 32, 0, st>>>(k0, nb, n, U, ldu, C, ldc, f);
        if (rest >= TRSS_TC_MIN) {
            // C_rr -= X^T U + U^T X on tensor cores: the SYRDK kernel on C's upper triangle
            if (launch_trss_split_tc(U, ldu, C, ldc, k0, nb, k1, (int)rest, out, f, limbs, opA, opB, st) !=
                cudaSuccess)
                return LDLT_ERR_CUDA;
            uint32_t *blk = C + k1 * ldc + k1;
            if (launch_syrdk_tc(blk, ldc, sigma, ls, out, opA, opB, limbs, f, blk, 2000000000LL, status, nsm, 0,
                                st, 1) != cudaSuccess)
                return LDLT_ERR_CUDA;
        } else {
            const unsigned gp = (unsigned)((rest + TC - 1) / TC);
            if (p >= (1u << 28))
                trss_syr2k_kernel<true><<<dim3(gp, gp), 256, 0, st>>>(k0, nb, n, U, ldu, C, ldc, f);
            else
                trss_syr2k_kernel<false><<<dim3(gp, gp), 256, 0, st>>>(k0, nb, n, U, ldu, C, ldc, f);
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
            trss_syr2k_kernel<true><<<dim3(gp, gp), 256, 0, st>>>(k0, nb, n, U, ldu, C, ldc, f);
        else
            trss_syr2k_kernel<false><<<dim3(gp, gp), 256, 0, st>>>(k0, nb, n, U, ldu, C, ldc, f);
    }
    return cudaGetLastError() == cudaSuccess ? LDLT_OK : LDLT_ERR_CUDA;
}
