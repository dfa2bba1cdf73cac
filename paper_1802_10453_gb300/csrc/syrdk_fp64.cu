// syrdk_fp64.cu -- FP64 form of the level-3 update of Algorithm 2:
//   Z = C - G D G^T   (SYRDK, Section 3), lower triangle only,
// written for the next Schur complement with the rows compacted (sigma).
//
// Residues are carried in doubles as balanced integers in (-p/2, p/2].  A
// product of two of them is at most ((p-1)/2)^2; blocks of kred products are
// summed exactly in FP64 and then reduced (r = acc - p*rint(acc/p), exact by
// FMA), so the running value stays below 2^53 while
//   kred * ((p-1)/2)^2 + 1.5 p < 2^53.
// That holds for kred >= 1 while p < 2^26.5; larger p is rejected on the host.
#include <cmath>

#include "ldlt_internal.cuh"

namespace {

constexpr int TB = 64;   // output tile TB x TB
constexpr int TK = 16;   // k chunk staged in shared memory

__device__ __forceinline__ double bal(uint32_t x, uint32_t p)
{
    return (double)(x > (p >> 1) ? (int64_t)x - (int64_t)p : (int64_t)x);
}

// GT[k][i] = G[i][k] = LpC[k][sigma[i]], GDT[k][i] = (G D)[i][k], balanced
// doubles; rows i >= m_next and columns np <= k < kpad are zero.
__global__ void split_fp64_kernel(const uint32_t *__restrict__ LpT, int64_t ldL,
                                  const int *__restrict__ sigma, const LoopState *__restrict__ ls,
                                  const PanelOut *__restrict__ out, FieldP f,
                                  double *__restrict__ GDT, double *__restrict__ GT, int64_t ldg,
                                  const uint32_t *__restrict__ S, int64_t ldS, uint32_t *__restrict__ Snext)
{
    if (!step_live(ls, out)) return;
    const int m_next = out->m_next, np = out->np;
    if (np == 0) {
        compact_rows(S, ldS, sigma, m_next, Snext, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
        return;
    }
    if (m_next == 0) return;
    const int kpad = (np + 63) / 64 * 64;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= (int)ldg || k >= kpad) return;
    double g = 0.0, gd = 0.0;
    if (i < m_next && k < np) {
        const int t = sigma[i];
        const uint32_t lk = LpT[(int64_t)k * ldL + t];
        uint32_t v;
        const uint32_t ek = out->eval[k];
        if (ek != 0) {
            v = fp_mul(ek, LpT[(int64_t)(k + 1) * ldL + t], f);
        } else if (k > 0 && out->eval[k - 1] != 0) {
            v = fp_add(fp_mul(out->eval[k - 1], LpT[(int64_t)(k - 1) * ldL + t], f),
                       fp_mul(out->dval[k], lk, f), f);
        } else {
            v = fp_mul(out->dval[k], lk, f);
        }
        g = bal(lk, f.p);
        gd = bal(v, f.p);
    }
    GT[(int64_t)k * ldg + i] = g;
    GDT[(int64_t)k * ldg + i] = gd;
}

__device__ __forceinline__ double red_p(double acc, double p, double pinv)
{
    return fma(-rint(acc * pinv), p, acc);
}

__device__ __forceinline__ void syrdk_fp64_tile(const uint32_t *__restrict__ S, int64_t ldS,
                                                const int *__restrict__ sigma, int m_next,
                                                const double *__restrict__ GDT, const double *__restrict__ GT,
                                                int64_t ldg, int kpad, int kred, FieldP f,
                                                uint32_t *__restrict__ Snext, int tIdx)
{
    // triangular tile index -> (I, J)
    int I = (int)((sqrt(8.0 * tIdx + 1.0) - 1.0) * 0.5);
    while ((I + 1) * (I + 2) / 2 <= tIdx) ++I;
    while (I * (I + 1) / 2 > tIdx) --I;
    const int J = tIdx - I * (I + 1) / 2;
    const int i0 = I * TB, j0 = J * TB;

    __shared__ double As[TK][TB];
    __shared__ double Bs[TK][TB];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const double p = (double)f.p, pinv = 1.0 / p;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    int cnt = 0;
    for (int k0 = 0; k0 < kpad; k0 += TK) {
        for (int q = threadIdx.x; q < TK * TB; q += 256) {
            int kk = q / TB, c = q % TB;
            As[kk][c] = GDT[(int64_t)(k0 + kk) * ldg + i0 + c];
            Bs[kk][c] = GT[(int64_t)(k0 + kk) * ldg + j0 + c];
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < TK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
            if (++cnt == kred) {
                cnt = 0;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = red_p(acc[a][b], p, pinv);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + ty + 16 * a;
        if (i >= m_next) continue;
        const uint32_t *srow = S + (int64_t)sigma[i] * ldS;
        uint32_t *drow = Snext + (int64_t)i * ldS;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + tx + 16 * b;
            if (j > i) continue;
            double r = red_p(acc[a][b], p, pinv);
            r -= p * floor(r * pinv);
            if (r < 0) r += p;
            if (r >= p) r -= p;
            const uint32_t dot = (uint32_t)r;
            drow[j] = fp_sub(srow[sigma[j]], dot, f);
        }
    }
}

// A CTA computes TB x TB tiles (I, J), J <= I, grid-strided, of
//   Snext[i][j] = S[sigma i][sigma j] - sum_k GD[i][k] G[j][k]   (i >= j).
__global__ void __launch_bounds__(256) syrdk_fp64_kernel(
    const uint32_t *__restrict__ S, int64_t ldS, const int *__restrict__ sigma,
    const LoopState *__restrict__ ls, const PanelOut *__restrict__ out,
    const double *__restrict__ GDT, const double *__restrict__ GT, int64_t ldg, int kred,
    FieldP f, uint32_t *__restrict__ Snext)
{
    if (!step_live(ls, out)) return;
    const int m_next = out->m_next, np = out->np;
    if (m_next == 0 || np == 0) return;
    const int kpad = (np + 63) / 64 * 64;
    const int nb = (m_next + TB - 1) / TB;
    const int ntiles = nb * (nb + 1) / 2;
    for (int tIdx = blockIdx.x; tIdx < ntiles; tIdx += gridDim.x)
        syrdk_fp64_tile(S, ldS, sigma, m_next, GDT, GT, ldg, kpad, kred, f, Snext, tIdx);
}

}  // namespace

size_t fp64_operand_bytes(int64_t n)
{
    const int64_t ldg = round_up(n, 64);
    return (size_t)2 * (size_t)KP_MAX * (size_t)ldg * sizeof(double);
}

cudaError_t launch_split_fp64(const uint32_t *LpC, int64_t ldL, const int *sigma, int64_t n,
                              const LoopState *ls, const PanelOut *out, FieldP f, double *GDT,
                              double *GT, int64_t ldg, const uint32_t *S, int64_t ldS, uint32_t *Snext,
                              cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    // sized for the largest update (ldg rows, KP_MAX columns); surplus threads return
    dim3 grid((unsigned)((ldg + 255) / 256), KP_MAX);
    split_fp64_kernel<<<grid, 256, 0, st>>>(LpC, ldL, sigma, ls, out, f, GDT, GT, ldg, S, ldS, Snext);
    return cudaGetLastError();
}

cudaError_t launch_syrdk_fp64(const uint32_t *S, int64_t ldS, const int *sigma, int64_t n,
                              const LoopState *ls, const PanelOut *out, const double *GDT,
                              const double *GT, int64_t ldg, FieldP f, uint32_t *Snext,
                              cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const double h = (double)((f.p - 1) / 2);
    const double lim = 9007199254740992.0 - 1.5 * (double)f.p;  // 2^53 - 1.5p
    int kred = (int)std::floor(lim / (h * h > 1.0 ? h * h : 1.0));
    if (kred > 1 << 20) kred = 1 << 20;
    if (kred < 1) return cudaErrorInvalidValue;
    const int64_t nb = (n + TB - 1) / TB;
    int64_t tiles = nb * (nb + 1) / 2;
    if (tiles > 4096) tiles = 4096;  // grid-strided over the tiles of the current order
    syrdk_fp64_kernel<<<(unsigned)tiles, 256, 0, st>>>(S, ldS, sigma, ls, out, GDT, GT, ldg, kred, f, Snext);
    return cudaGetLastError();
}
