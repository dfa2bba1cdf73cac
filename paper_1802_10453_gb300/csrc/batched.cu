// batched.cu -- the batched schedule: many independent small factorisations
// P^T A P = L D L^T mod p in one persistent launch.
//
// Every CTA takes whole matrices (order n <= BT_MAXN) from a queue sorted by
// decreasing n (longest first, so the tail of the launch is short) and factors
// one matrix at a time without leaving the SM:
//   ingest  -- S = lower(A) mod p, stored transposed (row a of S holds the
//              Schur column of row a contiguously), in the CTA's scratch;
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
// The CTAs never wait on one another: the only synchronisation is
// __syncthreads inside a CTA and one atomic counter for the queue.
#include <climits>
#include <cstddef>
#include <cstdint>

#include "../../include/ldlt_rpm.h"
#include "ldlt_internal.cuh"

namespace {

constexpr int BT_MAXN = 512;       // largest order of the batched schedule
constexpr int BT_THREADS = 256;    // 8 warps, rows tid and tid + 256
constexpr int BT_NWARP = BT_THREADS / 32;
constexpr int BT_NR = 4;           // S rows in flight on the pivot chain
constexpr int BT_TILE = 64;        // update tile
constexpr int BT_MAX_GRID = 640;   // CTAs at most (4 per SM on 152 SMs + slack)
constexpr size_t BT_CTA_WORDS = 2ull * BT_MAXN * BT_MAXN;  // S + Lw per CTA

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
};

template <int KB>
struct BtShared {
    static constexpr int LPS = KB + 1;  // odd row stride: conflict-free column reads
    uint32_t Lp[BT_MAXN * LPS];         // panel columns, raw (scaled) then normalised
    union {
        uint32_t ring[BT_NR][BT_MAXN];  // S rows prefetched for the pivot chain
        struct {
            uint32_t gd[BT_TILE * LPS]; // update: (G D) rows of the tile
            uint32_t gt[KB * BT_TILE];  // update: G columns of the tile, k-major
        } st;
        uint32_t tr[32 * 33];           // ingest transpose
    } u;
    int idx[BT_MAXN];                   // compact row -> original row
    int sig[BT_MAXN];                   // new compact row -> old compact row
    int plist[BT_MAXN];                 // pivot rows (original), pivot order
    uint32_t dv[BT_MAXN], ev[BT_MAXN];  // D diagonal, x at 2x2 block starts
    int zlist[BT_MAXN], zcnt[BT_MAXN];  // zero rows (original) and pivots before each
    uint32_t z[KB], z2[KB];             // z vectors of the current row (and partner)
    uint32_t wcol[KB];                  // w of each column's block (later pivots' product)
    uint32_t bx[KB], by[KB], bW[KB];    // scaled d (or x), scaled y, W before the block
    int role[KB];                       // 1: 1x1, 2: first / 3: second column of a 2x2
    uint32_t cinv[KB], cdel[KB];        // normalisation: 1/bx, scaled delta
    uint32_t tx[KB], ty[KB];            // true d (or x) and y of D, for G D
    unsigned char consumed[BT_MAXN];
    int fz[2 * BT_NWARP];
    int wsum[BT_NWARP];
    int mat;
};

__device__ __forceinline__ void bt_cp16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void bt_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bt_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <bool BIG>
__device__ __forceinline__ void bt_mac(uint64_t &acc, uint32_t a, uint32_t b, const FieldP &f)
{
    if (BIG) fp_mac(acc, a, b, f);
    else acc += (uint64_t)a * (uint64_t)b;  // p < 2^29: up to 64 terms stay below 2^64
}

// Row `row` of S (columns from row & ~3 up to m, in 16-byte pieces) -> slot.
__device__ __forceinline__ void bt_fetch_row(uint32_t *slot, const uint32_t *S, int ld, int row, int m,
                                             int tid)
{
    const int c0 = row & ~3;
    const int nq = (m - c0 + 3) >> 2;
    for (int q = tid; q < nq; q += BT_THREADS)
        bt_cp16(slot + c0 + 4 * q, S + (size_t)row * ld + c0 + 4 * q);
}

// z_k for the row `row`: entry k of concat_B w_B M_B U_B[row]^T, with M_B = 1
// for a 1x1 block and [[-y, x], [x, 0]] for a 2x2 block (scaled values).
template <int KB>
__device__ __forceinline__ uint32_t bt_zval(const BtShared<KB> &sh, int k, int row, const FieldP &f)
{
    const uint32_t *Lr = sh.Lp + row * BtShared<KB>::LPS;
    const int role = sh.role[k];
    uint32_t v;
    if (role == 1) v = Lr[k];
    else if (role == 2) v = fp_sub(fp_mul(sh.bx[k], Lr[k + 1], f), fp_mul(sh.by[k], Lr[k], f), f);
    else v = fp_mul(sh.bx[k], Lr[k - 1], f);
    return fp_mul(v, sh.wcol[k], f);
}

// c = W * s - sum_k U[t][k] z[k]  (the scaled Schur entry of row t)
template <int KB, bool BIG>
__device__ __forceinline__ uint32_t bt_schur(const uint32_t *Lt, const uint32_t *z, int np, uint32_t W,
                                             uint32_t s, const FieldP &f)
{
    uint64_t n0 = 0, n1 = 0;
    int k = 0;
    for (; k + 1 < np; k += 2) {
        bt_mac<BIG>(n0, Lt[k], z[k], f);
        bt_mac<BIG>(n1, Lt[k + 1], z[k + 1], f);
    }
    if (k < np) bt_mac<BIG>(n0, Lt[k], z[k], f);
    const uint32_t neg = fp_add(fp_reduce64(n0, f), fp_reduce64(n1, f), f);
    return fp_sub(fp_mul(W, s, f), neg, f);
}

template <int KB, bool BIG>
__global__ void __launch_bounds__(BT_THREADS, KB == 16 ? 3 : (KB == 32 ? 2 : 1)) batched_kernel(BatchParams P)
{
    extern __shared__ __align__(16) unsigned char bt_smem[];
    BtShared<KB> &sh = *reinterpret_cast<BtShared<KB> *>(bt_smem);
    constexpr int LPS = BtShared<KB>::LPS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FieldP f = P.f;
    uint32_t *const S = P.scratch + (size_t)blockIdx.x * BT_CTA_WORDS;
    uint32_t *const Lw = S + (size_t)BT_MAXN * BT_MAXN;

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
        const int ld = (n + 31) & ~31;
        const int kb = (n < P.ncut && P.kbsmall < KB) ? P.kbsmall : KB;

        // ---- ingest: S[j][i] = A[i][j] mod p for j <= i (32x32 transposes) ----
        for (int I = 0; I * 32 < n; ++I) {
            for (int J = 0; J <= I; ++J) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = I * 32 + warp + 8 * q, j = J * 32 + lane;
                    uint32_t v = 0;
                    if (i < n && j <= i) v = fp_reduce64((uint64_t)__ldcg(A + (size_t)i * lda + j), f);
                    sh.u.tr[(warp + 8 * q) * 33 + lane] = v;
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jr = J * 32 + warp + 8 * q, ic = I * 32 + lane;
                    if (ic < n && jr <= ic) S[(size_t)jr * ld + ic] = sh.u.tr[lane * 33 + warp + 8 * q];
                }
                __syncthreads();
            }
        }
        for (int t = tid; t < n; t += BT_THREADS) sh.idx[t] = t;

        int m = n, r0 = 0, nz = 0;
        while (m > 0) {
            // ---------------- panel: Crout pivot chain over the rows of S ----------------
            for (int t = tid; t < m; t += BT_THREADS) sh.consumed[t] = 0;
            __syncthreads();  // also orders the previous update's stores before the row copies
#pragma unroll
            for (int q = 0; q < BT_NR - 1; ++q) {
                if (q < m) bt_fetch_row(sh.u.ring[q], S, ld, q, m, tid);
                bt_commit();
            }
            int np = 0;
            uint32_t W = 1;
            int a = 0;
            bool full = false;
            for (; a < m && !full; ++a) {
                const int pre = a + BT_NR - 1;
                if (pre < m) bt_fetch_row(sh.u.ring[pre % BT_NR], S, ld, pre, m, tid);
                bt_commit();
                if (sh.consumed[a]) continue;  // partner of an earlier 2x2 pivot (uniform)
                bt_wait<BT_NR - 1>();
                if (tid < np) sh.z[tid] = bt_zval<KB>(sh, tid, a, f);
                __syncthreads();  // B1: z and row a of S visible

                const uint32_t *srow = sh.u.ring[a % BT_NR];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int t = tid + h * BT_THREADS;
                    bool nzf = false;
                    if (t >= a && t < m && !sh.consumed[t]) {
                        uint32_t *Lt = sh.Lp + t * LPS;
                        const uint32_t c = bt_schur<KB, BIG>(Lt, sh.z, np, W, srow[t], f);
                        Lt[np] = c;
                        nzf = (c != 0) && (t > a);
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, nzf);
                    if (lane == 0)
                        sh.fz[h * BT_NWARP + warp] = bal ? (h * BT_THREADS + warp * 32 + __ffs(bal) - 1) : INT_MAX;
                }
                __syncthreads();  // B2: column a of the Schur complement (scaled) complete

                const uint32_t caa = sh.Lp[a * LPS + np];
                if (caa != 0) {
                    // 1x1 pivot d = S_aa (Algorithm 4: non-zero diagonal)
                    if (tid < np) sh.wcol[tid] = fp_mul(sh.wcol[tid], caa, f);
                    if (tid == np) { sh.role[np] = 1; sh.wcol[np] = 1; sh.bx[np] = caa; sh.by[np] = 0; sh.bW[np] = W; }
                    if (tid == 0) sh.plist[r0 + np] = sh.idx[a];
                    W = fp_mul(W, caa, f);
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
                                sv[h] = __ldcg(S + (size_t)lo * ld + hi);
                            }
                        }
                        if (tid < np) sh.z2[tid] = bt_zval<KB>(sh, tid, b, f);
                        __syncthreads();  // B3
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int u = tid + h * BT_THREADS;
                            if (u >= a && u < m && !sh.consumed[u]) {
                                uint32_t *Lu = sh.Lp + u * LPS;
                                Lu[np + 1] = bt_schur<KB, BIG>(Lu, sh.z2, np, W, sv[h], f);
                            }
                        }
                        __syncthreads();  // B4
                        const uint32_t xt = sh.Lp[b * LPS + np], yt = sh.Lp[b * LPS + np + 1];
                        const uint32_t del = fp_mul(xt, xt, f);
                        if (tid < np) sh.wcol[tid] = fp_mul(sh.wcol[tid], del, f);
                        if (tid == np || tid == np + 1) {
                            sh.role[tid] = (tid == np) ? 2 : 3;
                            sh.wcol[tid] = 1; sh.bx[tid] = xt; sh.by[tid] = yt; sh.bW[tid] = W;
                        }
                        if (tid == 0) { sh.plist[r0 + np] = sh.idx[a]; sh.plist[r0 + np + 1] = sh.idx[b]; }
                        sh.consumed[b] = 1;  // every thread writes it: each sees its own store
                        W = fp_mul(W, del, f);
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
            bt_wait<0>();
            __syncthreads();  // no copy in flight, all pivots recorded

            // ---------------- normalise the panel's columns ----------------
            if (tid < np) {
                const int k = tid, role = sh.role[k];
                const uint32_t ix = fp_inv(sh.bx[k], f);
                const uint32_t iW = fp_inv(sh.bW[k], f);
                const uint32_t xtrue = fp_mul(sh.bx[k], iW, f);  // true d or x
                uint32_t ytrue = 0, dtil = 0;
                if (role != 1) {
                    ytrue = (f.p == 2) ? fp_mul(sh.by[k], iW, f) : 0u;      // y of D (p = 2 only)
                    dtil = (f.p == 2) ? sh.by[k] : fp_mul(sh.by[k], f.inv2, f);  // scaled delta
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
                            Lt[k] = fp_mul(Lt[k], sh.cinv[k], f);
                            k += 1;
                        } else {
                            // beta = U_a / x, alpha = (U_b - beta * delta) / x (scaled values)
                            const uint32_t ix = sh.cinv[k];
                            const uint32_t beta = fp_mul(Lt[k], ix, f);
                            const uint32_t alpha = fp_mul(fp_sub(Lt[k + 1], fp_mul(beta, sh.cdel[k], f), f), ix, f);
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
                uint32_t *dst = Lw + (size_t)sh.idx[t] * ld + r0;
                for (int k = lane; k < np; k += 32) dst[k] = sh.Lp[t * LPS + k];
            }

            // ---------------- rows left: sigma (ascending) ----------------
            const int t0 = 2 * tid;
            const int f0 = (t0 >= a_next && t0 < m && !sh.consumed[t0]) ? 1 : 0;
            const int f1 = (t0 + 1 >= a_next && t0 + 1 < m && !sh.consumed[t0 + 1]) ? 1 : 0;
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
                const int s = sh.wsum[w];
                if (w < warp) base += s;
                mn += s;
            }
            {
                int pos = base + incl - cnt;
                if (f0) sh.sig[pos++] = t0;
                if (f1) sh.sig[pos] = t0 + 1;
            }
            __syncthreads();

            // ---------------- update: S'[i][j] = S[sig i][sig j] - (G D G^T)[sig i][sig j] ----------------
            const int nt = (mn + BT_TILE - 1) / BT_TILE;
            const int tx = tid & 15, ty = tid >> 4;
            for (int I = 0; I < nt; ++I) {
                for (int J = I; J < nt; ++J) {
                    uint32_t old[4][4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int i = I * BT_TILE + ty * 4 + q;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int j = J * BT_TILE + tx + 16 * c;
                            old[q][c] = (i < mn && j < mn && i <= j)
                                            ? __ldcg(S + (size_t)sh.sig[i] * ld + sh.sig[j]) : 0u;
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
                                if (role == 1) v = fp_mul(sh.tx[k], Lt[k], f);
                                else if (role == 2) v = fp_mul(sh.tx[k], Lt[k + 1], f);
                                else v = fp_add(fp_mul(sh.tx[k], Lt[k - 1], f), fp_mul(sh.ty[k], Lt[k], f), f);
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
                            if (i < mn && j < mn && i <= j)
                                S[(size_t)i * ld + j] = fp_sub(old[q][c], fp_reduce64(acc[q][c], f), f);
                        }
                    }
                    __syncthreads();
                }
            }
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
            const uint32_t *Lr = Lw + (size_t)src * ld;
            for (int j = lane; j <= k; j += 32) Ak[j] = (j == k) ? dk : (j < cmax ? __ldcg(Lr + j) : 0u);
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

template <int KB, bool BIG>
cudaError_t bt_launch(const BatchParams &P, int grid_cap, int nsm, cudaStream_t st)
{
    const size_t smem = sizeof(BtShared<KB>);
    auto kern = batched_kernel<KB, BIG>;
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

    if (cudaMemsetAsync(w + L.next, 0, sizeof(int), st) != cudaSuccess) return LDLT_ERR_CUDA;
    bt_order_kernel<<<1, 1024, 0, st>>>(n, count, (int *)(w + L.order));
    if (cudaGetLastError() != cudaSuccess) return LDLT_ERR_CUDA;
    const bool big = p >= (1u << 29);
    cudaError_t err;
    if (g_bt_kb == 16) err = big ? bt_launch<16, true>(P, grid_cap, nsm, st) : bt_launch<16, false>(P, grid_cap, nsm, st);
    else if (g_bt_kb == 64) err = big ? bt_launch<64, true>(P, grid_cap, nsm, st) : bt_launch<64, false>(P, grid_cap, nsm, st);
    else err = big ? bt_launch<32, true>(P, grid_cap, nsm, st) : bt_launch<32, false>(P, grid_cap, nsm, st);
    return err == cudaSuccess ? LDLT_OK : LDLT_ERR_CUDA;
}
