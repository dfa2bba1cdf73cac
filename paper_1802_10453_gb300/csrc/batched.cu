// batched.cu -- the batched schedule: many independent small factorisations
// P^T A P = L D L^T mod p in one persistent launch.
//
// Every CTA takes whole matrices (order n <= BT_MAXN) from a queue sorted by
// decreasing n (longest first, so the tail of the launch is short) and factors
// one matrix at a time without leaving the SM.  The Schur complement S lives
// in the lower triangle of the caller's A itself (compacted to the leading
// rows as pivots leave); the CTA's scratch only holds L by original row.
//   panel   -- the lexicographic pivot search of Algorithm 4 (Section 5), row
//              by row, in Crout form over at most kb pivots.  All remaining
//              rows of the matrix are in the CTA, so the test for a zero row
//              and the search for the first non-zero partner are a CTA-wide
//              ballot.  Columns are kept scaled by the product W of the
//              panel's pivot determinants (no division on the pivot chain)
//              and are normalised once per panel;
//   update  -- S <- S[sigma, sigma] - G D G^T on the rows left (the SYRDK
//              step of Algorithm 2, Section 4), 64x64 tiles on CUDA cores,
//              rows compacted in place;
//   finalize-- A <- L in pivot order with D on the diagonal.
// Entries of the input are reduced mod p when the first panel reads them.
// The CTAs never wait on one another: the only synchronisation is
// __syncthreads inside a CTA and one atomic counter for the queue.
#include <climits>
#include <cstddef>
#include <cstdint>

#include <cuda_bf16.h>

#include "../../include/ldlt_rpm.h"
#include "ldlt_internal.cuh"

namespace {

constexpr int BT_MAXN = 512;       // largest order of the batched schedule
constexpr int BT_THREADS = 256;    // 8 warps, rows tid and tid + 256
constexpr int BT_NWARP = BT_THREADS / 32;
constexpr int BT_NR = 4;           // S columns in flight on the pivot chain
constexpr int BT_TILE = 64;        // update tile
constexpr int BT_MAX_GRID = 640;   // CTAs at most (4 per SM on 152 SMs + slack)
constexpr size_t BT_CTA_WORDS = (size_t)BT_MAXN * BT_MAXN;  // L by original row, per CTA

int g_bt_kb = 32;       // panel width the kernel is compiled for (16, 32, 64)
int g_bt_ncut = 0;      // orders below this use g_bt_kbsmall
int g_bt_kbsmall = 32;

struct BatchParams {
    int64_t count;
    const int64_t *n;
    const int64_t *lda;
    uint32_t *const *A;
    int32_t *const *perm;
    uint32_t *const *e;
    int64_t *rank;
    int32_t *status;
    FieldP f;
    const int *order;
    int *next;
    uint32_t *scratch;
    int ncut, kbsmall;
    uint32_t mu32, c32;  // floor(2^32 / p), 2^32 mod p (used when p < 2^16)
};

// Field operations of the batched kernel: the generic 64-bit forms of
// field.cuh, or for p < 2^16 (residue products below 2^32) Barrett
// reductions on 32-bit words.
template <bool P16>
struct BtField {
    FieldP f;
    uint32_t mu32, c32;
    __device__ __forceinline__ uint32_t red32(uint32_t x) const
    {
        const uint32_t q = __umulhi(x, mu32);  // floor(x / p) or one less
        const uint32_t r = x - q * f.p;
        return r >= f.p ? r - f.p : r;
    }
    __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) const
    {
        if constexpr (P16) return red32(a * b);
        else return fp_mul(a, b, f);
    }
    // x mod p; for p < 2^16 valid for x < 2^47 (hi * (2^32 mod p) + p < 2^32)
    __device__ __forceinline__ uint32_t red(uint64_t x) const
    {
        if constexpr (P16) return red32((uint32_t)(x >> 32) * c32 + red32((uint32_t)x));
        else return fp_reduce64(x, f);
    }
};

template <int KB>
struct BtShared {
    static constexpr int LPS = KB + 1;  // odd row stride: conflict-free column reads
    uint32_t Lp[BT_MAXN * LPS];         // panel columns, raw (scaled) then normalised
    union {
        uint32_t ring[BT_NR][BT_MAXN];  // S columns prefetched for the pivot chain
        struct {
            uint32_t gd[BT_TILE * LPS]; // update: (G D) rows of the tile
            uint32_t gt[KB * BT_TILE];  // update: G columns of the tile, k-major
        } st;
        struct {                        // tensor-core update: bf16 limb pairs, K contiguous
            uint32_t a[2][BT_TILE][(KB + 8) / 2];  // limbs of (G D) rows of the tile
            uint32_t b[2][BT_TILE][(KB + 8) / 2];  // limbs of G rows of the tile's columns
        } mt;
    } u;
    int idx[BT_MAXN];                   // compact row -> original row
    int sig[BT_MAXN];                   // new compact row -> old compact row
    int plist[BT_MAXN];                 // pivot rows (original), pivot order
    uint32_t dv[BT_MAXN], ev[BT_MAXN];  // D diagonal, x at 2x2 block starts
    int zlist[BT_MAXN], zcnt[BT_MAXN];  // zero rows (original) and pivots before each
    uint32_t z[KB], z2[KB];             // -z vectors of the current row (and partner)
    uint32_t cw1[KB], cw2[KB];          // z coefficients: w (1x1), w x and w y (2x2)
    uint32_t bx[KB], by[KB], bW[KB];    // scaled d (or x), scaled y, W before the block
    int role[KB];                       // 1: 1x1, 2: first / 3: second column of a 2x2
    uint32_t cinv[KB], cdel[KB];        // normalisation: 1/bx, scaled delta
    uint32_t tx[KB], ty[KB];            // true d (or x) and y of D, for G D
    unsigned char consumed[BT_MAXN];
    int fz[2 * BT_NWARP];
    int wsum[BT_NWARP];
    int mat;
};

template <bool BIG>
__device__ __forceinline__ void bt_mac(uint64_t &acc, uint32_t a, uint32_t b, const FieldP &f)
{
    if (BIG) fp_mac(acc, a, b, f);
    else acc += (uint64_t)a * (uint64_t)b;  // p < 2^28: 65 terms stay below 2^63
}

// Column a of S below the diagonal (lower storage): the entries of the
// thread's two rows, loaded from L2 (never through L1: the update rewrites S
// in place, and an L1 copy of a line could be stale).
__device__ __forceinline__ void bt_load_col(uint32_t &v0, uint32_t &v1, const uint32_t *S, int64_t ld, int a,
                                            int m, int t0, int t1)
{
    v0 = (t0 >= a && t0 < m) ? __ldcg(S + (size_t)t0 * ld + a) : 0u;
    v1 = (t1 >= a && t1 < m) ? __ldcg(S + (size_t)t1 * ld + a) : 0u;
}

// -z_k for the row `row`: entry k of concat_B w_B M_B U_B[row]^T, negated,
// with M_B = 1 for a 1x1 block and [[-y, x], [x, 0]] for a 2x2 block (scaled
// values; the coefficients w, w x, w y are kept per column).
template <int KB, bool P16>
__device__ __forceinline__ uint32_t bt_negz(const BtShared<KB> &sh, int k, int row, const BtField<P16> &F)
{
    const uint32_t *Lr = sh.Lp + row * BtShared<KB>::LPS;
    const int role = sh.role[k];
    uint32_t v;
    if (role == 1) v = F.mul(sh.cw1[k], Lr[k]);
    else if (role == 2) v = fp_sub(F.mul(sh.cw1[k], Lr[k + 1]), F.mul(sh.cw2[k], Lr[k]), F.f);
    else v = F.mul(sh.cw1[k], Lr[k - 1]);
    return v ? F.f.p - v : 0u;
}

// Scaled Schur entries W s_h + sum_k U[t_h][k] (-z_k) of the thread's two rows.
template <int KB, bool BIG, bool P16>
__device__ __forceinline__ void bt_schur2(const uint32_t *L0, const uint32_t *L1, const uint32_t *nz, int np,
                                          uint32_t W, uint32_t s0, uint32_t s1, const BtField<P16> &F,
                                          uint32_t &c0, uint32_t &c1)
{
    uint64_t a0 = (uint64_t)W * s0, a1 = (uint64_t)W * s1;
#pragma unroll 4
    for (int k = 0; k < np; ++k) {
        const uint32_t zk = nz[k];
        bt_mac<BIG>(a0, L0[k], zk, F.f);
        bt_mac<BIG>(a1, L1[k], zk, F.f);
    }
    c0 = F.red(a0);
    c1 = F.red(a1);
}

// Balanced residue of x in two signed 8-bit limbs: bal(x) = d0 + 256 d1 with
// d0 in [-128, 127] and |d1| <= 128 (enough for (p - 1) / 2 <= 128 + 128 * 256), each limb
// exact in bf16.  Returns the two limbs' bf16 bit patterns in the low halves.
constexpr uint32_t BT_MMA_PMAX = 65535;  // p < 2^16: two limbs, 32-bit field words

__device__ __forceinline__ void bt_limbs2(uint32_t x, uint32_t p, uint32_t &l0, uint32_t &l1)
{
    const int v = (x > (p >> 1)) ? (int)x - (int)p : (int)x;
    const int d0 = (int)(signed char)(v & 0xFF);
    const int d1 = (v - d0) >> 8;
    l0 = __bfloat16_as_ushort(__float2bfloat16_rn((float)d0));
    l1 = __bfloat16_as_ushort(__float2bfloat16_rn((float)d1));
}

// D (16x8, f32) += A (16x16, bf16, row) * B (16x8, bf16, col): one warp.
__device__ __forceinline__ void bt_mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int KB, bool BIG, bool MMA>
__global__ void __launch_bounds__(BT_THREADS, KB == 16 ? 3 : (KB == 32 ? 2 : 1)) batched_kernel(BatchParams P)
{
    extern __shared__ __align__(16) unsigned char bt_smem[];
    BtShared<KB> &sh = *reinterpret_cast<BtShared<KB> *>(bt_smem);
    constexpr int LPS = BtShared<KB>::LPS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FieldP f = P.f;
    BtField<MMA> F;
    F.f = P.f;
    F.mu32 = P.mu32;
    F.c32 = P.c32;
    uint32_t *const Lw = P.scratch + (size_t)blockIdx.x * BT_CTA_WORDS;

    for (;;) {
        if (tid == 0) {
            const int i = atomicAdd(P.next, 1);
            sh.mat = (i < P.count) ? P.order[i] : -1;
        }
        __syncthreads();
        const int mat = sh.mat;
        if (mat < 0) return;

        const int64_t n64 = P.n[mat];
        const int64_t lda = P.lda[mat];
        uint32_t *const A = P.A[mat];
        int32_t *const perm = P.perm[mat];
        uint32_t *const eo = P.e[mat];
        if (n64 < 0 || n64 > BT_MAXN || (n64 > 0 && (lda < n64 || !A || !perm || !eo))) {
            if (tid == 0) { P.status[mat] = LDLT_ERR_ARG; P.rank[mat] = 0; }
            __syncthreads();
            continue;
        }
        const int n = (int)n64;
        if (n == 0) {
            if (tid == 0) { P.status[mat] = LDLT_OK; P.rank[mat] = 0; }
            __syncthreads();
            continue;
        }
        uint32_t *const S = A;                  // lower triangle, leading dimension lda
        const int ldw = (n + 31) & ~31;         // Lw row stride
        const int kb = (n < P.ncut && P.kbsmall < KB) ? P.kbsmall : KB;
        for (int t = tid; t < n; t += BT_THREADS) sh.idx[t] = t;

        int m = n, r0 = 0, nz = 0;
        bool raw = true;  // S still holds input entries (not yet reduced mod p)
        while (m > 0) {
            // ---------------- panel: Crout pivot chain over the rows of S ----------------
            for (int t = tid; t < m; t += BT_THREADS) sh.consumed[t] = 0;
            __syncthreads();  // also orders the previous update's stores before the column loads
            const int t0 = tid, t1 = tid + BT_THREADS;
            // Columns of S run ahead of the chain: column a+2 is in the thread's
            // ring slots (each thread reads back only its own two entries) and
            // column a+3 is in flight in registers.
#pragma unroll
            for (int q = 0; q < BT_NR - 1; ++q) {
                if (q < m) {
                    uint32_t v0, v1;
                    bt_load_col(v0, v1, S, lda, q, m, t0, t1);
                    sh.u.ring[q][t0] = v0;
                    sh.u.ring[q][t1] = v1;
                }
            }
            uint32_t pf0 = 0, pf1 = 0;
            int pf_col = -1;
            int np = 0;
            uint32_t W = 1;
            int a = 0;
            bool full = false;
            for (; a < m && !full; ++a) {
                if (pf_col >= 0) {
                    sh.u.ring[pf_col % BT_NR][t0] = pf0;
                    sh.u.ring[pf_col % BT_NR][t1] = pf1;
                }
                pf_col = a + BT_NR - 1;
                if (pf_col < m) bt_load_col(pf0, pf1, S, lda, pf_col, m, t0, t1);
                else pf_col = -1;
                if (sh.consumed[a]) continue;  // partner of an earlier 2x2 pivot (uniform)
                if (tid < np) sh.z[tid] = bt_negz<KB, MMA>(sh, tid, a, F);
                __syncthreads();  // B1: z visible

                const uint32_t *scol = sh.u.ring[a % BT_NR];
                const bool v0 = t0 >= a && t0 < m && !sh.consumed[t0];
                const bool v1 = t1 >= a && t1 < m && !sh.consumed[t1];
                uint32_t s0 = v0 ? scol[t0] : 0u, s1 = v1 ? scol[t1] : 0u;
                if (raw) { s0 = F.red(s0); s1 = F.red(s1); }
                uint32_t c0, c1;
                bt_schur2<KB, BIG, MMA>(sh.Lp + t0 * LPS, sh.Lp + t1 * LPS, sh.z, np, W, s0, s1, F, c0, c1);
                if (v0) sh.Lp[t0 * LPS + np] = c0;
                if (v1) sh.Lp[t1 * LPS + np] = c1;
                {
                    const unsigned b0 = __ballot_sync(0xffffffffu, v0 && c0 != 0 && t0 > a);
                    const unsigned b1 = __ballot_sync(0xffffffffu, v1 && c1 != 0 && t1 > a);
                    if (lane == 0) {
                        sh.fz[warp] = b0 ? (warp * 32 + __ffs(b0) - 1) : INT_MAX;
                        sh.fz[BT_NWARP + warp] = b1 ? (BT_THREADS + warp * 32 + __ffs(b1) - 1) : INT_MAX;
                    }
                }
                __syncthreads();  // B2: column a of the Schur complement (scaled) complete

                const uint32_t caa = sh.Lp[a * LPS + np];
                if (caa != 0) {
                    // 1x1 pivot d = S_aa (Algorithm 4: non-zero diagonal)
                    if (tid < np) {
                        sh.cw1[tid] = F.mul(sh.cw1[tid], caa);
                        if (sh.role[tid] == 2) sh.cw2[tid] = F.mul(sh.cw2[tid], caa);
                    }
                    if (tid == np) {
                        sh.role[np] = 1; sh.cw1[np] = 1; sh.cw2[np] = 0;
                        sh.bx[np] = caa; sh.by[np] = 0; sh.bW[np] = W;
                    }
                    if (tid == 0) sh.plist[r0 + np] = sh.idx[a];
                    W = F.mul(W, caa);
                    np += 1;
                } else {
                    int b = INT_MAX;
#pragma unroll
                    for (int q = 0; q < 2 * BT_NWARP; ++q) b = min(b, sh.fz[q]);
                    if (b < m) {
                        // 2x2 pivot on (a, b), b the first non-zero of row a (Algorithm 4)
                        uint32_t sv[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int u = tid + h * BT_THREADS;
                            sv[h] = 0;
                            if (u >= a && u < m && !sh.consumed[u]) {
                                const int lo = min(u, b), hi = max(u, b);
                                sv[h] = __ldcg(S + (size_t)hi * lda + lo);
                                if (raw) sv[h] = F.red(sv[h]);
                            }
                        }
                        if (tid < np) sh.z2[tid] = bt_negz<KB, MMA>(sh, tid, b, F);
                        __syncthreads();  // B3
                        uint32_t d0, d1;
                        bt_schur2<KB, BIG, MMA>(sh.Lp + t0 * LPS, sh.Lp + t1 * LPS, sh.z2, np, W, sv[0], sv[1], F, d0, d1);
                        if (v0) sh.Lp[t0 * LPS + np + 1] = d0;
                        if (v1) sh.Lp[t1 * LPS + np + 1] = d1;
                        __syncthreads();  // B4
                        const uint32_t xt = sh.Lp[b * LPS + np], yt = sh.Lp[b * LPS + np + 1];
                        const uint32_t del = F.mul(xt, xt);
                        if (tid < np) {
                            sh.cw1[tid] = F.mul(sh.cw1[tid], del);
                            if (sh.role[tid] == 2) sh.cw2[tid] = F.mul(sh.cw2[tid], del);
                        }
                        if (tid == np || tid == np + 1) {
                            sh.role[tid] = (tid == np) ? 2 : 3;
                            sh.cw1[tid] = xt; sh.cw2[tid] = (tid == np) ? yt : 0u;
                            sh.bx[tid] = xt; sh.by[tid] = yt; sh.bW[tid] = W;
                        }
                        if (tid == 0) { sh.plist[r0 + np] = sh.idx[a]; sh.plist[r0 + np + 1] = sh.idx[b]; }
                        sh.consumed[b] = 1;  // every thread writes it: each sees its own store
                        W = F.mul(W, del);
                        np += 2;
                    } else {
                        // row a of the Schur complement is zero: not a pivot row
                        if (tid == 0) { sh.zlist[nz] = sh.idx[a]; sh.zcnt[nz] = r0 + np; }
                        nz += 1;
                    }
                }
                full = np > kb - 2;
            }
            const int a_next = a;
            __syncthreads();  // all pivots recorded

            // ---------------- normalise the panel's columns ----------------
            if (tid < np) {
                const int k = tid, role = sh.role[k];
                const uint32_t ix = fp_inv(sh.bx[k], f);
                const uint32_t iW = fp_inv(sh.bW[k], f);
                const uint32_t xtrue = F.mul(sh.bx[k], iW);  // true d or x
                uint32_t ytrue = 0, dtil = 0;
                if (role != 1) {
                    ytrue = (f.p == 2) ? F.mul(sh.by[k], iW) : 0u;           // y of D (p = 2 only)
                    dtil = (f.p == 2) ? sh.by[k] : F.mul(sh.by[k], f.inv2);  // scaled delta
                }
                sh.cinv[k] = ix; sh.cdel[k] = dtil;
                sh.tx[k] = xtrue; sh.ty[k] = ytrue;
                const int pos = r0 + k;
                if (role == 1) { sh.dv[pos] = xtrue; sh.ev[pos] = 0; }
                else if (role == 2) { sh.dv[pos] = 0; sh.ev[pos] = xtrue; }
                else { sh.dv[pos] = ytrue; sh.ev[pos] = 0; }
            }
            __syncthreads();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = tid + h * BT_THREADS;
                if (t < m) {
                    uint32_t *Lt = sh.Lp + t * LPS;
                    for (int k = 0; k < np;) {
                        if (sh.role[k] == 1) {
                            Lt[k] = F.mul(Lt[k], sh.cinv[k]);
                            k += 1;
                        } else {
                            // beta = U_a / x, alpha = (U_b - beta * delta) / x (scaled values)
                            const uint32_t ix = sh.cinv[k];
                            const uint32_t beta = F.mul(Lt[k], ix);
                            const uint32_t alpha = F.mul(fp_sub(Lt[k + 1], F.mul(beta, sh.cdel[k]), f), ix);
                            Lt[k] = alpha;
                            Lt[k + 1] = beta;
                            k += 2;
                        }
                    }
                }
            }
            __syncthreads();
            // L columns r0 .. r0+np-1 of every row of this panel, by original row
            for (int t = warp; t < m; t += BT_NWARP) {
                uint32_t *dst = Lw + (size_t)sh.idx[t] * ldw + r0;
                for (int k = lane; k < np; k += 32) dst[k] = sh.Lp[t * LPS + k];
            }

            // ---------------- rows left: sigma (ascending) ----------------
            const int u0 = 2 * tid;
            const int f0 = (u0 >= a_next && u0 < m && !sh.consumed[u0]) ? 1 : 0;
            const int f1 = (u0 + 1 >= a_next && u0 + 1 < m && !sh.consumed[u0 + 1]) ? 1 : 0;
            const int cnt = f0 + f1;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) sh.wsum[warp] = incl;
            __syncthreads();
            int base = 0, mn = 0;
#pragma unroll
            for (int w = 0; w < BT_NWARP; ++w) {
                const int sw = sh.wsum[w];
                if (w < warp) base += sw;
                mn += sw;
            }
            {
                int pos = base + incl - cnt;
                if (f0) sh.sig[pos++] = u0;
                if (f1) sh.sig[pos] = u0 + 1;
            }
            __syncthreads();

            // ---------------- update: S'[i][j] = S[sig i][sig j] - (G D G^T)[sig i][sig j], i >= j ----------------
            // Tiles in row-major order over the lower triangle: every read of a
            // later tile lies in a row or column beyond what earlier tiles wrote.
            const int nt = (mn + BT_TILE - 1) / BT_TILE;
            if constexpr (MMA) {
                // Tensor-core form: bal(x) = d0 + 256 d1 for both operands, so
                // (GD) G^T = sum_w 256^w acc_w with acc_0 = A0 B0^T,
                // acc_1 = A0 B1^T + A1 B0^T, acc_2 = A1 B1^T over bf16 limbs;
                // |acc_w| <= 2 * 64 * 128^2 < 2^24, exact in f32.
                constexpr int KW = (KB + 8) / 2;
                const int ksteps = (np + 15) >> 4;
                const int kw2 = (np + 1) >> 1;  // limb pairs holding data
                const int g = lane >> 2, tig = lane & 3;
                const int wm = warp >> 1, wn = warp & 1;  // 16 rows x 32 columns per warp
                // |acc_0|, |acc_2| <= 64 * 128^2 = 2^20 and |acc_1| <= 2^21: multiples of p
                // that make the two partial sums non-negative and below 2^32
                const int off30 = (int)(((1u << 30) / f.p + 1) * f.p);
                const int off22 = (int)(((1u << 21) / f.p + 1) * f.p);
                for (int I = 0; I < nt; ++I) {
                    for (int J = 0; J <= I; ++J) {
                        const int rbase = I * BT_TILE + wm * 16 + g;
                        const int cbase = J * BT_TILE + wn * 32 + 2 * tig;
                        uint32_t old[2][4][2];
#pragma unroll
                        for (int hr = 0; hr < 2; ++hr) {
                            const int i = rbase + 8 * hr;
#pragma unroll
                            for (int nf = 0; nf < 4; ++nf)
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    const int j = cbase + nf * 8 + e;
                                    // consumed only in the epilogue: the load stays in flight
                                    old[hr][nf][e] = (i < mn && j <= i)
                                                         ? __ldcg(S + (size_t)sh.sig[i] * lda + sh.sig[j]) : 0u;
                                }
                        }
                        if (J == 0) {
                            // limbs of the (G D) rows of row block I (k pairs)
#pragma unroll
                            for (int it = 0; it < BT_TILE * KW / BT_THREADS; ++it) {
                                const int q = tid + it * BT_THREADS;
                                const int rr = q / KW, kp = q - rr * KW;
                                const int tn = I * BT_TILE + rr;
                                uint32_t w0 = 0, w1 = 0;
                                if (tn < mn && kp < kw2) {
                                    const uint32_t *Lt = sh.Lp + sh.sig[tn] * LPS;
#pragma unroll
                                    for (int e = 0; e < 2; ++e) {
                                        const int k = 2 * kp + e;
                                        uint32_t v = 0;
                                        if (k < np) {
                                            const int role = sh.role[k];
                                            if (role == 1) v = F.mul(sh.tx[k], Lt[k]);
                                            else if (role == 2) v = F.mul(sh.tx[k], Lt[k + 1]);
                                            else v = fp_add(F.mul(sh.tx[k], Lt[k - 1]), F.mul(sh.ty[k], Lt[k]), f);
                                        }
                                        uint32_t l0, l1;
                                        bt_limbs2(v, f.p, l0, l1);
                                        w0 |= l0 << (16 * e);
                                        w1 |= l1 << (16 * e);
                                    }
                                }
                                sh.u.mt.a[0][rr][kp] = w0;
                                sh.u.mt.a[1][rr][kp] = w1;
                            }
                        }
                        // limbs of the G rows of column block J
#pragma unroll
                        for (int it = 0; it < BT_TILE * KW / BT_THREADS; ++it) {
                            const int q = tid + it * BT_THREADS;
                            const int cc = q / KW, kp = q - cc * KW;
                            const int tn = J * BT_TILE + cc;
                            uint32_t w0 = 0, w1 = 0;
                            if (tn < mn && kp < kw2) {
                                const uint32_t *Lt = sh.Lp + sh.sig[tn] * LPS;
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    const int k = 2 * kp + e;
                                    uint32_t l0, l1;
                                    bt_limbs2(k < np ? Lt[k] : 0u, f.p, l0, l1);
                                    w0 |= l0 << (16 * e);
                                    w1 |= l1 << (16 * e);
                                }
                            }
                            sh.u.mt.b[0][cc][kp] = w0;
                            sh.u.mt.b[1][cc][kp] = w1;
                        }
                        __syncthreads();
                        float acc[3][4][4];
#pragma unroll
                        for (int w = 0; w < 3; ++w)
#pragma unroll
                            for (int nf = 0; nf < 4; ++nf)
#pragma unroll
                                for (int e = 0; e < 4; ++e) acc[w][nf][e] = 0.f;
                        const int ar = wm * 16 + g;
                        for (int ks = 0; ks < ksteps; ++ks) {
                            const int kw = ks * 8 + tig;
                            uint32_t af[2][4];
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                af[u][0] = sh.u.mt.a[u][ar][kw];
                                af[u][1] = sh.u.mt.a[u][ar + 8][kw];
                                af[u][2] = sh.u.mt.a[u][ar][kw + 4];
                                af[u][3] = sh.u.mt.a[u][ar + 8][kw + 4];
                            }
#pragma unroll
                            for (int nf = 0; nf < 4; ++nf) {
                                const int bc = wn * 32 + nf * 8 + g;
                                uint32_t bf[2][2];
#pragma unroll
                                for (int v = 0; v < 2; ++v) {
                                    bf[v][0] = sh.u.mt.b[v][bc][kw];
                                    bf[v][1] = sh.u.mt.b[v][bc][kw + 4];
                                }
                                bt_mma(acc[0][nf], af[0], bf[0][0], bf[0][1]);
                                bt_mma(acc[1][nf], af[0], bf[1][0], bf[1][1]);
                                bt_mma(acc[1][nf], af[1], bf[0][0], bf[0][1]);
                                bt_mma(acc[2][nf], af[1], bf[1][0], bf[1][1]);
                            }
                        }
#pragma unroll
                        for (int hr = 0; hr < 2; ++hr) {
                            const int i = rbase + 8 * hr;
#pragma unroll
                            for (int nf = 0; nf < 4; ++nf)
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    const int j = cbase + nf * 8 + e;
                                    if (i < mn && j <= i) {
                                        // sum_w 256^w acc_w mod p in two 32-bit steps
                                        const int ci = 2 * hr + e;
                                        const int a0 = __float2int_rn(acc[0][nf][ci]);
                                        const int a1 = __float2int_rn(acc[1][nf][ci]);
                                        const int a2 = __float2int_rn(acc[2][nf][ci]);
                                        const uint32_t hi = F.red32((uint32_t)(a1 + 256 * a2 + off30));
                                        const uint32_t prod = F.red32((uint32_t)(a0 + 256 * (int)hi + off22));
                                        const uint32_t ov = raw ? F.red32(old[hr][nf][e]) : old[hr][nf][e];
                                        S[(size_t)i * lda + j] = fp_sub(ov, prod, f);
                                    }
                                }
                        }
                        __syncthreads();
                    }
                }
            } else {
                const int tx = tid & 15, ty = tid >> 4;
                for (int I = 0; I < nt; ++I) {
                    for (int J = 0; J <= I; ++J) {
                        uint32_t old[4][4];
    #pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int i = I * BT_TILE + ty * 4 + q;
    #pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int j = J * BT_TILE + tx + 16 * c;
                                old[q][c] = (i < mn && j <= i) ? __ldcg(S + (size_t)sh.sig[i] * lda + sh.sig[j]) : 0u;
                            }
                        }
                        for (int rr = warp; rr < BT_TILE; rr += BT_NWARP) {
                            const int tn = I * BT_TILE + rr;
                            const int t = tn < mn ? sh.sig[tn] : -1;
                            for (int k = lane; k < np; k += 32) {
                                uint32_t v = 0;
                                if (t >= 0) {
                                    const uint32_t *Lt = sh.Lp + t * LPS;
                                    const int role = sh.role[k];
                                    if (role == 1) v = F.mul(sh.tx[k], Lt[k]);
                                    else if (role == 2) v = F.mul(sh.tx[k], Lt[k + 1]);
                                    else v = fp_add(F.mul(sh.tx[k], Lt[k - 1]), F.mul(sh.ty[k], Lt[k]), f);
                                }
                                sh.u.st.gd[rr * LPS + k] = v;
                            }
                        }
                        for (int k = warp; k < np; k += BT_NWARP) {
                            for (int c = lane; c < BT_TILE; c += 32) {
                                const int tn = J * BT_TILE + c;
                                sh.u.st.gt[k * BT_TILE + c] = tn < mn ? sh.Lp[sh.sig[tn] * LPS + k] : 0u;
                            }
                        }
                        __syncthreads();
                        uint64_t acc[4][4];
    #pragma unroll
                        for (int q = 0; q < 4; ++q)
    #pragma unroll
                            for (int c = 0; c < 4; ++c) acc[q][c] = 0;
                        for (int k = 0; k < np; ++k) {
                            uint32_t g[4], hh[4];
    #pragma unroll
                            for (int q = 0; q < 4; ++q) g[q] = sh.u.st.gd[(ty * 4 + q) * LPS + k];
    #pragma unroll
                            for (int c = 0; c < 4; ++c) hh[c] = sh.u.st.gt[k * BT_TILE + tx + 16 * c];
    #pragma unroll
                            for (int q = 0; q < 4; ++q)
    #pragma unroll
                                for (int c = 0; c < 4; ++c) bt_mac<BIG>(acc[q][c], g[q], hh[c], f);
                        }
    #pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int i = I * BT_TILE + ty * 4 + q;
    #pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int j = J * BT_TILE + tx + 16 * c;
                                if (i < mn && j <= i)
                                    S[(size_t)i * lda + j] =
                                        fp_sub(raw ? F.red(old[q][c]) : old[q][c], F.red(acc[q][c]), f);
                            }
                        }
                        __syncthreads();
                    }
                }
            }
            raw = false;
            // compact the original-index map
            int ni[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = tid + h * BT_THREADS;
                ni[h] = t < mn ? sh.idx[sh.sig[t]] : 0;
            }
            __syncthreads();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = tid + h * BT_THREADS;
                if (t < mn) sh.idx[t] = ni[h];
            }
            r0 += np;
            m = mn;
            __syncthreads();
        }

        // ---------------- finalize: A <- L (pivot order) with D on the diagonal ----------------
        const int r = r0;
        for (int k = tid; k < n; k += BT_THREADS) {
            perm[k] = k < r ? sh.plist[k] : sh.zlist[k - r];
            eo[k] = k < r ? sh.ev[k] : 0u;
        }
        for (int k = warp; k < n; k += BT_NWARP) {
            const int src = k < r ? sh.plist[k] : sh.zlist[k - r];
            const int cmax = k < r ? k : sh.zcnt[k - r];
            const uint32_t dk = k < r ? sh.dv[k] : 0u;
            uint32_t *Ak = A + (size_t)k * lda;
            const uint32_t *Lr = Lw + (size_t)src * ldw;
            for (int j0 = 0; j0 <= k; j0 += 128) {
                uint32_t v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = j0 + lane + 32 * q;
                    v[q] = (j < k && j < cmax) ? __ldcg(Lr + j) : 0u;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = j0 + lane + 32 * q;
                    if (j <= k) Ak[j] = (j == k) ? dk : v[q];
                }
            }
        }
        if (tid == 0) { P.rank[mat] = r; P.status[mat] = LDLT_OK; }
        __syncthreads();
    }
}

// Queue order: matrices by decreasing n (invalid orders first: they finish at
// once).  One CTA, counting sort over n in [0, BT_MAXN].
constexpr int BT_KEYS = BT_MAXN + 2;

__global__ void __launch_bounds__(1024) bt_order_kernel(const int64_t *n, int64_t count, int *order)
{
    __shared__ int cnt[BT_KEYS];
    for (int k = threadIdx.x; k < BT_KEYS; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    auto key = [&](int64_t i) {
        const int64_t v = n[i];
        return (v < 0 || v > BT_MAXN) ? 0 : (int)(BT_MAXN - v) + 1;
    };
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) atomicAdd(&cnt[key(i)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int k = 0; k < BT_KEYS; ++k) { const int c = cnt[k]; cnt[k] = s; s += c; }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) order[atomicAdd(&cnt[key(i)], 1)] = (int)i;
}

struct BtLayout {
    size_t next, order, scratch, header;
};

BtLayout bt_layout(int64_t count)
{
    BtLayout L;
    L.next = 0;
    L.order = 256;
    L.scratch = L.order + (size_t)round_up(count * 4, 256);
    L.header = L.scratch;
    return L;
}

template <int KB, bool BIG, bool MMA>
cudaError_t bt_launch(const BatchParams &P, int grid_cap, int nsm, cudaStream_t st)
{
    const size_t smem = sizeof(BtShared<KB>);
    auto kern = batched_kernel<KB, BIG, MMA>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT_THREADS, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * nsm;
    if (grid > grid_cap) grid = grid_cap;
    if (grid > P.count) grid = P.count;
    if (grid < 1) grid = 1;
    kern<<<(int)grid, BT_THREADS, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace

extern "C" int ldlt_rpm_batched_workspace_bytes(int64_t count, uint32_t p, int path, size_t *bytes)
{
    if (!bytes || count < 0 || count > INT_MAX) return LDLT_ERR_ARG;
    size_t tmp = 0;
    const int rc = ldlt_rpm_workspace_bytes(1, p, path, &tmp);  // p and path checks
    if (rc != LDLT_OK) return rc;
    const BtLayout L = bt_layout(count);
    const int64_t ncta = count < BT_MAX_GRID ? count : BT_MAX_GRID;
    *bytes = L.header + (size_t)ncta * BT_CTA_WORDS * 4;
    return LDLT_OK;
}

extern "C" int ldlt_rpm_batched_set_schedule(int kb, int n_cut, int kb_small)
{
    if (kb != 16 && kb != 32 && kb != 64) return LDLT_ERR_ARG;
    if (n_cut < 0 || n_cut > BT_MAXN + 1) return LDLT_ERR_ARG;
    if (kb_small < 4 || kb_small > kb) return LDLT_ERR_ARG;
    g_bt_kb = kb;
    g_bt_ncut = n_cut;
    g_bt_kbsmall = kb_small;
    return LDLT_OK;
}

extern "C" int ldlt_rpm_factor_batched(int64_t count, const int64_t *n, uint32_t p, uint32_t *const *A,
                                       const int64_t *lda, int32_t *const *perm, uint32_t *const *e,
                                       int64_t *rank, int32_t *status, int path, void *ws, size_t ws_bytes,
                                       void *stream)
{
    if (count < 0 || count > INT_MAX) return LDLT_ERR_ARG;
    size_t tmp = 0;
    int rc = ldlt_rpm_workspace_bytes(1, p, path, &tmp);
    if (rc != LDLT_OK) return rc;
    if (count == 0) return LDLT_OK;
    if (!n || !A || !lda || !perm || !e || !rank || !status) return LDLT_ERR_ARG;
    const BtLayout L = bt_layout(count);
    if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < L.header + BT_CTA_WORDS * 4) return LDLT_ERR_WORKSPACE;
    const int64_t fit = (int64_t)((ws_bytes - L.header) / (BT_CTA_WORDS * 4));
    const int grid_cap = (int)(fit < BT_MAX_GRID ? fit : BT_MAX_GRID);

    int dev = 0, major = 0, minor = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDLT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LDLT_ERR_CUDA;
    if (major != 10 || minor != 3) return LDLT_ERR_NO_DEVICE;

    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *w = (uint8_t *)ws;
    BatchParams P;
    P.count = count; P.n = n; P.lda = lda; P.A = A; P.perm = perm; P.e = e;
    P.rank = rank; P.status = status; P.f = make_field(p);
    P.order = (const int *)(w + L.order);
    P.next = (int *)(w + L.next);
    P.scratch = (uint32_t *)(w + L.scratch);
    P.ncut = g_bt_ncut; P.kbsmall = g_bt_kbsmall;
    P.mu32 = (uint32_t)((1ull << 32) / p);
    P.c32 = (uint32_t)((1ull << 32) % p);

    if (cudaMemsetAsync(w + L.next, 0, sizeof(int), st) != cudaSuccess) return LDLT_ERR_CUDA;
    bt_order_kernel<<<1, 1024, 0, st>>>(n, count, (int *)(w + L.order));
    if (cudaGetLastError() != cudaSuccess) return LDLT_ERR_CUDA;
    // exact integer arithmetic: for p < 2^16 32-bit field words and the
    // tensor-core update with two bf16 limbs, else 64-bit words and the
    // CUDA-core update
    const int form = p <= BT_MMA_PMAX ? 0 : (p < (1u << 28) ? 1 : 2);
    cudaError_t err;
    if (g_bt_kb == 16)
        err = form == 0 ? bt_launch<16, false, true>(P, grid_cap, nsm, st)
            : form == 1 ? bt_launch<16, false, false>(P, grid_cap, nsm, st)
                        : bt_launch<16, true, false>(P, grid_cap, nsm, st);
    else if (g_bt_kb == 64)
        err = form == 0 ? bt_launch<64, false, true>(P, grid_cap, nsm, st)
            : form == 1 ? bt_launch<64, false, false>(P, grid_cap, nsm, st)
                        : bt_launch<64, true, false>(P, grid_cap, nsm, st);
    else
        err = form == 0 ? bt_launch<32, false, true>(P, grid_cap, nsm, st)
            : form == 1 ? bt_launch<32, false, false>(P, grid_cap, nsm, st)
                        : bt_launch<32, true, false>(P, grid_cap, nsm, st);
    return err == cudaSuccess ? LDLT_OK : LDLT_ERR_CUDA;
}
