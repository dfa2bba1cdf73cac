// gen_kernels.cu -- GPU form of the seeded input generator of inputs.py.
//
// Holds none of the factorisation's arithmetic and shares no code with it: it
// draws the same matrices as the host generator (checked by the tests), fast
// enough for orders in the tens of thousands.
//   planted:  A = T R T^T mod p with T[i][k] = uniform(key_T, i*n + k) below the
//             diagonal, 1 on it; R given as a list of terms (k_q, p_q, s_q),
//             A[i][j] = sum_q T[i][k_q] s_q T[j][p_q].
//   uniform:  A[i][j] = uniform(key_U, max(i,j)*n + min(i,j)).
// Only the lower triangle (with the diagonal) of A is written.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t uniform_mod(uint64_t key, uint64_t ctr, uint32_t p)
{
    uint64_t out = mix64(key + (ctr + 1ull) * 0x9E3779B97F4A7C15ull);
    return (uint32_t)(((out >> 32) * (uint64_t)p) >> 32);
}

__device__ __forceinline__ uint32_t t_entry(uint64_t key, int64_t n, int64_t i, int64_t k, uint32_t p)
{
    if (k > i) return 0u;
    if (k == i) return 1u;
    return uniform_mod(key, (uint64_t)(i * n + k), p);
}

// TkT[q][i] = T[i][k_q];  TpT[q][j] = s_q T[j][p_q] mod p.
__global__ void gen_factors_kernel(int64_t n, uint32_t p, uint64_t keyT, int nterms, int64_t ldt,
                                   const int *__restrict__ kq, const int *__restrict__ pq,
                                   const uint32_t *__restrict__ sq, uint32_t *__restrict__ TkT,
                                   uint32_t *__restrict__ TpT)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (q >= nterms) return;
    if (i >= ldt) return;
    uint32_t a = 0, b = 0;
    if (i < n) {
        a = t_entry(keyT, n, i, kq[q], p);
        b = (uint32_t)(((uint64_t)t_entry(keyT, n, i, pq[q], p) * sq[q]) % p);
    }
    TkT[(int64_t)q * ldt + i] = a;
    TpT[(int64_t)q * ldt + i] = b;
}

// A[i][j] = sum_q TkT[q][i] TpT[q][j] mod p for j <= i, 64 x 64 tiles.
__global__ void __launch_bounds__(256) gen_product_kernel(int64_t n, uint32_t p, int nterms, int64_t ldt,
                                                          const uint32_t *__restrict__ TkT,
                                                          const uint32_t *__restrict__ TpT,
                                                          uint32_t *__restrict__ A, int64_t lda)
{
    const int64_t tIdx = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)tIdx + 1.0) - 1.0) * 0.5);
    while ((I + 1) * (I + 2) / 2 <= tIdx) ++I;
    while (I * (I + 1) / 2 > tIdx) --I;
    const int64_t J = tIdx - I * (I + 1) / 2;
    const int64_t i0 = I * 64, j0 = J * 64;
    __shared__ uint32_t As[16][64], Bs[16][64];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const uint64_t pp = (uint64_t)p * p;
    const uint64_t big = ((1ull << 63) / pp) * pp;  // multiple of p in (2^62, 2^63]
    uint64_t acc[4][4] = {};
    for (int q0 = 0; q0 < nterms; q0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int kk = e / 64, c = e % 64;
            bool ok = q0 + kk < nterms;
            As[kk][c] = ok ? TkT[(int64_t)(q0 + kk) * ldt + i0 + c] : 0u;
            Bs[kk][c] = ok ? TpT[(int64_t)(q0 + kk) * ldt + j0 + c] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    uint64_t s = acc[a][b] + (uint64_t)As[kk][ty + 16 * a] * Bs[kk][tx + 16 * b];
                    acc[a][b] = s - (s >> 63) * big;
                }
        }
        __syncthreads();
    }
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + ty + 16 * a;
        if (i >= n) continue;
        for (int b = 0; b < 4; ++b) {
            const int64_t j = j0 + tx + 16 * b;
            if (j > i) continue;
            A[i * lda + j] = (uint32_t)(acc[a][b] % p);
        }
    }
}

__global__ void gen_uniform_kernel(int64_t n, uint32_t p, uint64_t keyU, uint32_t *__restrict__ A, int64_t lda)
{
    const int64_t i = blockIdx.y;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= i; j += (int64_t)gridDim.x * blockDim.x)
        A[i * lda + j] = uniform_mod(keyU, (uint64_t)(i * n + j), p);
}

}  // namespace

extern "C" {

// Workspace for ldlt_gen_planted: 2 * nterms * round_up(n, 64) * 4 bytes.
size_t ldlt_gen_planted_ws_bytes(int64_t n, int nterms)
{
    const int64_t ldt = (n + 63) / 64 * 64;
    return (size_t)2 * (size_t)(nterms > 0 ? nterms : 1) * (size_t)ldt * 4;
}

int ldlt_gen_planted(int64_t n, uint32_t p, uint64_t keyT, int nterms, const int *kq, const int *pq,
                     const uint32_t *sq, uint32_t *A, int64_t lda, void *ws, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (n <= 0) return 0;
    const int64_t ldt = (n + 63) / 64 * 64;
    const int64_t nb = (n + 63) / 64;
    if (nterms == 0) {
        for (int64_t i = 0; i < n; ++i)
            if (cudaMemsetAsync(A + i * lda, 0, (size_t)(i + 1) * 4, st) != cudaSuccess) return -5;
        return 0;
    }
    uint32_t *TkT = (uint32_t *)ws;
    uint32_t *TpT = TkT + (int64_t)nterms * ldt;
    dim3 g1((unsigned)((ldt + 255) / 256), (unsigned)nterms);
    gen_factors_kernel<<<g1, 256, 0, st>>>(n, p, keyT, nterms, ldt, kq, pq, sq, TkT, TpT);
    gen_product_kernel<<<(unsigned)(nb * (nb + 1) / 2), 256, 0, st>>>(n, p, nterms, ldt, TkT, TpT, A, lda);
    return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

int ldlt_gen_uniform(int64_t n, uint32_t p, uint64_t keyU, uint32_t *A, int64_t lda, void *stream)
{
    if (n <= 0) return 0;
    dim3 g((unsigned)((n + 255) / 256 > 64 ? 64 : (n + 255) / 256), (unsigned)n);
    gen_uniform_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(n, p, keyU, A, lda);
    return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

}  // extern "C"
