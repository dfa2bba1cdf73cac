// panel.cu -- the pivot chain: one panel of the lexicographic elimination.
//
// Dumas & Pernet, Algorithm 4 (Section 5).  Rows of the current Schur
// complement S are visited in ascending order.  Row a becomes
//   * a 1x1 pivot if its diagonal entry c_a[a] is non-zero;
//   * a 2x2 pivot with b, the first index > a with c_a[b] != 0;
//   * a non-pivot row if its Schur row is zero.
// c_a[t] = S[t][a] - sum_k L[t][k] (D L[a])_k is the Crout form of the Schur
// entry (the "c <- A_{i..n,i} - N v^T" step of Algorithm 4, with D in place of
// the printed D^{-1}).
//
// Division-free form.  A modular inverse is a long serial computation; taking
// one per pivot on the decision path would dominate the chain.  The panel
// therefore keeps, for every row t, the unscaled Schur columns U~[t][k] and,
// per pivot block B, an integer 2x2 (or 1x1) form M_B and a non-zero
// "denominator" delta_B such that the block's share of the Crout sum is
//   U~[t][B] M_B U~[a][B]^T / delta_B.
// With W = prod_B delta_B and w_B = W / delta_B (both kept by multiplication
// only) the scaled Schur entry is
//   c~_a[t] = W c_a[t] = W S[t][a] - sum_k U~[t][k] z_a[k],
//   z_a = concat_B  M_B U~[a][B]^T w_B,
// and c~ is zero exactly when c is.  A 1x1 pivot stores U~[:, j] = c~_a
// (M = 1, delta = W c~_a[a]); a 2x2 pivot stores c~_a and c~_b
// (M = [[-y~, x~], [x~, 0]], delta = W x~^2, x~ = c~_a[b], y~ = c~_b[b]).  The
// block forms follow from Algorithm 4's 2x2 branch: with beta = c_a / x,
// alpha = (c_b - delta' beta) / x and D = [[0,x],[x,y']], the product
// [alpha, beta] D [alpha', beta']^T equals [c_a, c_b] [[-y/x^2, 1/x],[1/x, 0]]
// [c_a', c_b']^T for both odd p (y' = 0, delta' = y/2) and p = 2 (y' = delta'
// = y).  At the end of the panel all inverses are taken at once (Montgomery's
// batch inversion) and every CTA rewrites its U~ rows as the true L columns;
// D is reported in true values.  The results are identical to the divided
// form because all arithmetic is exact.
//
// GPU organisation.  One cooperative launch per panel.  CTA 0 (the leader)
// owns the window of the first W rows of S and takes every decision.  The
// other CTAs (helpers) own the far rows [W, m) in contiguous slices.  Each CTA
// keeps the U~ columns of its rows in shared memory (k-major, padded) and
// writes them through to global memory.  16 compute warps work two threads
// per row.  In the leader, warp 17 publishes events to the helpers from a
// shared-memory ring so the gpu-scope fence stays off the critical path; in a
// helper, warp 16 prefetches events into the ring.  Helpers compute the new
// columns of their rows as pivots are published and answer "far scans": when
// a row has no non-zero inside the window, every helper searches its slice
// for the first non-zero of that row and the leader takes the minimum.  Every
// wait is bounded by a %globaltimer budget; when it runs out the kernel
// writes LDLT_ERR_TIMEOUT to the status word, raises an abort flag the other
// CTAs poll, and returns.
//
// At the end the leader compacts the remaining rows (order preserved) into
// sigma / idx_next for the next Schur complement.
#include <climits>

#include "ldlt_internal.cuh"

#define LDLT_ERR_TIMEOUT_CODE (-6)

// Cycle counters of the pivot chain (leader phases, helper idle time): built
// only with -DLDLT_CHAIN_PROFILE, so the release kernel reads no clock on its
// critical path.  The event and rollback counts are kept in every build.
#ifdef LDLT_CHAIN_PROFILE
#define CHAIN_PROF(...) __VA_ARGS__
#else
#define CHAIN_PROF(...)
#endif

namespace {

constexpr int NCW = 16;                       // compute warps
constexpr int NCT = NCW * 32;                 // compute threads (2 per row)
constexpr int SROWS = 256;                    // rows held in shared memory per CTA
constexpr int RS = KP_MAX + 8;                // U~ row stride (words): 8 mod 32, so the 16-byte
                                              // loads of 4 consecutive rows x 2 k-groups of a
                                              // quarter warp hit distinct banks
constexpr int NSLOT = 8;                      // event ring slots
constexpr int BLOCK = PANEL_THREADS_V2;

static_assert(BLOCK == NCT + 64, "two service warps");
static_assert(W0 <= SROWS && ROWS_PER_HELPER <= SROWS, "rows fit in shared memory");

enum ColKind : uint8_t { K_1x1 = 1, K_2A = 2, K_2B = 3 };

__device__ __forceinline__ int64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (int64_t)t;
}

// Budget check for spin-waits that reads %globaltimer only once every 1024
// unsuccessful spins (the first read starts the clock), so a wait that is
// already satisfied costs nothing.
struct Spin {
    int64_t t0 = 0;
    unsigned n = 0;
    __device__ __forceinline__ bool expired(int64_t budget)
    {
        if ((++n & 1023u) != 0) return false;
        const int64_t t = gtime();
        if (t0 == 0) { t0 = t; return false; }
        return t - t0 > budget;
    }
};

__device__ __forceinline__ uint32_t pick4(const uint4 &v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// barrier among the 16 compute warps only
__device__ __forceinline__ void cbar() { asm volatile("bar.sync 1, %0;" ::"n"(NCT) : "memory"); }

__device__ __forceinline__ uint32_t s_at(const uint32_t *__restrict__ S, int64_t ldS, int i, int j)
{
    return i >= j ? __ldg(S + (int64_t)i * ldS + j) : __ldg(S + (int64_t)j * ldS + i);
}

template <bool BIG>
__device__ __forceinline__ void mac(uint64_t &acc, uint32_t a, uint32_t b, const FieldP &f)
{
    acc += (uint64_t)a * (uint64_t)b;
    if (BIG) acc -= (acc >> 63) * f.m63;
}

constexpr int NPEND = 16;                     // speculative far scans in flight
// The far-scan bookkeeping (issue, answers, rollback requests) runs on the
// last compute warp, which holds no z entry (np <= KP_MAX <= CTL), so it
// overlaps the z vector of the first warps.  Its lane 0 (CTL) alone writes the
// pend_* records; between barriers only that warp reads them.
constexpr int CTL = NCT - 32;
static_assert(KP_MAX <= CTL, "the control thread computes no z entry");
constexpr int SRING = 128;                    // posted scan results

struct Shared {
    uint32_t U[SROWS * RS];            // U~ of this CTA's rows, row-major
    uint32_t ring[NSLOT][EV_WORDS];    // event payloads
    uint32_t scol[NSLOT][2][SROWS];    // helpers: S(t, a) and S(t, b) of each ring event
    uint4 sgrp[2][SROWS];              // helpers: S[t][4g .. 4g+3] for two column groups
    Event ev[NSLOT];
    uint32_t ub[KP_MAX];               // U~ row of a 2x2 partner
    uint8_t kind[KP_MAX];              // column kinds of this panel
    uint32_t bw[KP_MAX];               // w_B, at the block's first column
    uint32_t mx[KP_MAX], my[KP_MAX];   // x~, y~ of a 2x2 block (first column)
    uint32_t piv[KP_MAX];              // c~_a[a] (1x1) or x~ (2x2) at the first column
    uint32_t w0[KP_MAX];               // W when the block was formed
    uint32_t cA[KP_MAX], cB[KP_MAX];   // true-L coefficients (end of panel)
    uint32_t dtrue[KP_MAX], etrue[KP_MAX];
    uint32_t bi[2 * KP_MAX];           // batch inversion: values, then their inverses
    uint32_t bpre[2 * KP_MAX];         // batch inversion: prefix products
    int piv_rows[KP_MAX];
    int zero_rows[W0];
    int zero_np[W0];
    uint8_t wstate[W0];
    // speculative far scans: a row whose window part is zero is taken as a
    // zero row while its scan is in flight; a scan that finds a partner rolls
    // the panel back to that row.
    int pend_id[NPEND], pend_row[NPEND], pend_np[NPEND], pend_nz[NPEND];
    uint32_t pend_W[NPEND];
    uint32_t pend_bw[NPEND][KP_MAX];   // w_B when the scan was issued
    uint32_t delta[KP_MAX];            // delta_B at the block's first column
    int res_min[SRING];
    volatile int res_ok[SRING];        // id + 1 once scan id's answer is in res_min
    int redi[32];
    uint32_t xy[4];
    uint32_t caa;
    volatile int ev_ready;             // events written to the ring (leader) / fetched (helper)
    volatile int ev_done;              // events published (leader) / processed (helper)
    volatile int quit;
    volatile int ev_fetched;           // helpers: event records fetched (poller -> column loader)
    volatile int nscan_pub;            // scans published (leader -> watcher warp)
    uint32_t W;
    int np, ia, nzero, nscan, abort, b, owner, nblk;
    int ph_new, rb, rb_b;              // posted by the control warp: pending head, rollback request
    int nrollback;
    long long dbg[16];                 // diagnostics (thread-0 / lane-0 owned slots)
    int hgo;                           // helpers: the next event is in the ring (tid 0's decision)
};

// load with acquire semantics at GPU scope: later reads of this thread see
// every write that was made visible before the matching release / fence
__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// relaxed load at GPU scope: a flag read that a later fence can turn into an
// acquire
__device__ __forceinline__ unsigned ld_relaxed(const void *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// acquire load at CTA scope, for flags in shared memory: the "memory" clobber
// also keeps the compiler from hoisting later loads above it
__device__ __forceinline__ int ld_acquire_cta(const volatile int *p)
{
    int v;
    asm volatile("ld.acquire.cta.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ void raise_timeout(const PanelParams &P)
{
    atomicExch(P.status, LDLT_ERR_TIMEOUT_CODE);
    atomicExch(&P.sync->abort, 1);
}

// z[k] of row u (u read with a stride): M_B U~[u][B]^T w_B per block.
__device__ __forceinline__ uint32_t zval(int k, const uint32_t *u, int stride, const Shared &sh, const FieldP &f)
{
    const uint8_t kd = sh.kind[k];
    const int kb = k - (kd == K_2B);               // the block's first column
    const int j = k + (kd == K_2A) - (kd == K_2B);
    const uint32_t c1 = kd == K_1x1 ? 1u : sh.mx[kb];
    const uint32_t c2 = kd == K_2A ? sh.my[k] : 0u;
    const uint32_t t = fp_sub(fp_mul(c1, u[j * stride], f), fp_mul(c2, u[k * stride], f), f);
    return fp_mul(t, sh.bw[kb], f);
}

// c~_z[t] = W S(t, a) - sum_{k < np} U~[t][k] z[k], two threads per row.  In
// shared memory (row-major) half = tid & 1 takes the k-groups 8j + 4 half ..
// +3 with 16-byte loads of the row and of z (z is 16-byte aligned and zero
// from np to the next multiple of 8); rows kept in
// global memory (k-major) take every other k.  All 32 lanes must call it
// (pair shuffle); invalid rows compute nothing and return 0.
template <bool BIG>
__device__ __forceinline__ uint32_t schur2(const PanelParams &P, const uint32_t *sU, int lrow, int grow,
                                          uint32_t sval, uint32_t W, const uint32_t *z, int np, int half,
                                          bool valid, bool in_smem)
{
    uint64_t acc = 0;
    if (valid) {
        if (in_smem) {
            const uint4 *row = reinterpret_cast<const uint4 *>(sU + lrow * RS + 4 * half);
            const uint4 *zv = reinterpret_cast<const uint4 *>(z + 4 * half);
            const int ng = (np + 7) >> 3;
#pragma unroll 2
            for (int j = 0; j < ng; ++j) {
                const uint4 u = row[2 * j], zz = zv[2 * j];
                mac<BIG>(acc, u.x, zz.x, P.f);
                mac<BIG>(acc, u.y, zz.y, P.f);
                mac<BIG>(acc, u.z, zz.z, P.f);
                mac<BIG>(acc, u.w, zz.w, P.f);
            }
        } else {
            const uint32_t *col = P.LpT + grow;
            for (int k = half; k < np; k += 2) mac<BIG>(acc, col[(int64_t)k * P.ldL], z[k], P.f);
        }
    }
    const uint32_t part = fp_reduce64(acc, P.f);
    const uint32_t other = __shfl_xor_sync(0xffffffffu, part, 1);
    if (!valid) return 0u;
    return fp_sub(fp_mul(W, sval, P.f), fp_add(part, other, P.f), P.f);
}

// Rewrite the U~ values of one row as true L values into the output LpC (in
// global memory), using the per-column coefficients: 1x1: L_j = cA_j U_j; first column of a 2x2:
// L_j = cA_j U_{j+1} + cB_j U_j; second column: L_j = cA_j U_{j-1}.
__device__ __forceinline__ void finish_row(const PanelParams &P, const uint32_t *u, int stride, uint32_t *g,
                                           int np, const uint8_t *kind, const uint32_t *cA, const uint32_t *cB)
{
    for (int j = 0; j < np; ++j) {
        const uint8_t kd = kind[j];
        if (kd == K_1x1) {
            g[(int64_t)j * P.ldL] = fp_mul(cA[j], u[j * stride], P.f);
        } else if (kd == K_2A) {
            const uint32_t u0 = u[j * stride], u1 = u[(j + 1) * stride];
            g[(int64_t)j * P.ldL] = fp_add(fp_mul(cA[j], u1, P.f), fp_mul(cB[j], u0, P.f), P.f);
            g[(int64_t)(j + 1) * P.ldL] = fp_mul(cA[j + 1], u0, P.f);
            ++j;
        }
    }
}

// ---------------------------------------------------------------------------
// helper CTAs
// ---------------------------------------------------------------------------
template <bool BIG>
__device__ void helper_cta(const PanelParams &P, Shared &sh, int lo, int hi)
{
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nrows = hi > lo ? hi - lo : 0;
    if (tid == 0) { sh.ev_ready = 0; sh.ev_done = 0; sh.quit = 0; sh.ev_fetched = 0; }
    {
        const int nz = (nrows < SROWS ? nrows : SROWS) * RS / 4;
        for (int i = tid; i < nz; i += blockDim.x) reinterpret_cast<uint4 *>(sh.U)[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();

    if (warp == NCW) {
        // ---- poller: fetch every published event that fits into the ring ----
        int e = 0;
        for (;;) {
            int avail = 0;
            if (lane == 0) {
                Spin sp;
                volatile int *ab = &P.sync->abort;
                for (;;) {
                    const int c = ld_acquire(&P.sync->ev_count);
                    const int room = sh.ev_done + NSLOT;
                    const int lim = c < room ? c : room;
                    if (lim > e) { avail = lim - e; break; }
                    if (*ab) break;
                    if (sp.expired(P.budget_ns)) { raise_timeout(P); break; }
                }
            }
            avail = __shfl_sync(0xffffffffu, avail, 0);
            if (!avail) {
                if (lane == 0) { __threadfence_block(); sh.quit = 1; }
                return;
            }
            __syncwarp();  // lane 0's acquire of the count orders the record reads of the warp
            bool end = false;
            for (int q = 0; q < avail; ++q) {
                // one round trip: header and the first 2*KP_MAX payload words
                const int ee = e + q, s = ee % NSLOT;
                const uint4 *rec = reinterpret_cast<const uint4 *>(P.evlog + (int64_t)ee * EV_REC);
                constexpr int NCH = (8 + 2 * KP_MAX) / 4;
                uint4 c0 = __ldcg(rec + lane), c1 = __ldcg(rec + lane + 32), c2 = make_uint4(0, 0, 0, 0);
                if (lane + 64 < NCH) c2 = __ldcg(rec + lane + 64);
                uint4 *ringv = reinterpret_cast<uint4 *>(sh.ring[s]);
                uint4 *evv = reinterpret_cast<uint4 *>(&sh.ev[s]);
                if (lane < 2) evv[lane] = c0; else ringv[lane - 2] = c0;
                ringv[lane + 30] = c1;
                if (lane + 64 < NCH) ringv[lane + 62] = c2;
                const int kind = __shfl_sync(0xffffffffu, (int)c0.x, 0);
                if (kind == EV_END) {
                    // the end record carries 3*KP_MAX payload words
                    for (int k = 2 * KP_MAX / 4 + lane; k < 3 * KP_MAX / 4; k += 32)
                        ringv[k] = __ldcg(rec + 2 + k);
                    end = true;
                }
            }
            __threadfence_block();
            __syncwarp();
            if (lane == 0) sh.ev_fetched = e + avail;
            if (end) return;
            e += avail;
        }
    }
    if (warp == NCW + 1) {
        // ---- column loader: S(t, a) (and S(t, b)) of each fetched event for this CTA's rows ----
        // Columns come in groups of four (16-byte rows of S) kept in shared
        // memory; the next group is fetched with cp.async while the current
        // one serves events, so most events cost a shared-memory copy.
        const int nr = nrows < SROWS ? nrows : SROWS;
        int gbuf_g[2] = {-1, -1};
        int last_g = -1;  // group of the most recent cp.async commit
        auto fetch_grp = [&](int g, int bi) {
            for (int lr = lane; lr < nr; lr += 32) {
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&sh.sgrp[bi][lr]);
                const uint32_t *src = P.S + (int64_t)(lo + lr) * P.ldS + 4 * g;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            gbuf_g[bi] = g;
        };
        for (int e = 0;; ++e) {
            int go = 0;
            if (lane == 0) {
                Spin sp;
                for (;;) {
                    if (sh.ev_fetched > e) { go = 1; break; }
                    if (sh.quit) break;
                    __nanosleep(16);
                    if (sp.expired(2 * P.budget_ns + 1000000)) break;
                }
            }
            go = __shfl_sync(0xffffffffu, go, 0);
            if (!go) break;
            __threadfence_block();
            const int s = e % NSLOT;
            const int kind = sh.ev[s].kind, ea = sh.ev[s].a, eb = sh.ev[s].b;
            if (kind == EV_PIVOT1 || kind == EV_PIVOT2 || kind == EV_SCAN) {
                const int g = ea >> 2;
                int bi = (gbuf_g[0] == g) ? 0 : ((gbuf_g[1] == g) ? 1 : -1);
                if (bi < 0) {
                    // not resident (first event, or the row index went back): fetch now
                    asm volatile("cp.async.wait_group 0;" ::: "memory");
                    __syncwarp();
                    bi = (gbuf_g[0] == g + 1) ? 1 : 0;
                    fetch_grp(g, bi);
                    last_g = g;
                }
                // group g was committed before a later prefetch unless it is the last commit
                if (last_g == g) asm volatile("cp.async.wait_group 0;" ::: "memory");
                else asm volatile("cp.async.wait_group 1;" ::: "memory");
                __syncwarp();
                // t > a for every far row t: column a of row t
                const int c = ea & 3;
                for (int lr = lane; lr < nr; lr += 32) sh.scol[s][0][lr] = pick4(sh.sgrp[bi][lr], c);
                if (kind == EV_PIVOT2) {
                    // S(t, b): for t > b one line per row, so all loads of the
                    // lane go out before the first store (one round trip)
                    uint32_t v[SROWS / 32];
#pragma unroll
                    for (int i = 0; i < SROWS / 32; ++i) {
                        const int lr = lane + 32 * i;
                        v[i] = lr < nr ? s_at(P.S, P.ldS, lo + lr, eb) : 0u;
                    }
#pragma unroll
                    for (int i = 0; i < SROWS / 32; ++i)
                        if (lane + 32 * i < nr) sh.scol[s][1][lane + 32 * i] = v[i];
                }
                __syncwarp();
                if (gbuf_g[bi ^ 1] != g + 1) {
                    // prefetch the next group into the other buffer once nothing is in flight
                    if (last_g != g) asm volatile("cp.async.wait_group 0;" ::: "memory");
                    __syncwarp();
                    fetch_grp(g + 1, bi ^ 1);
                    last_g = g + 1;
                }
            }
            __threadfence_block();
            __syncwarp();
            if (lane == 0) sh.ev_ready = e + 1;
            if (kind == EV_END) break;
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        return;
    }
    // ---- compute warps ----
    const int half = tid & 1;
    CHAIN_PROF(long long hidle = 0, hbusy = 0, hmark = clock64();)
    auto hflush = [&]() {
        if (tid == 0 && blockIdx.x == 1) {
            CHAIN_PROF(P.out->dbg[5] = hidle; P.out->dbg[6] = hbusy;)
        }
    };
    for (int e = 0;; ++e) {
        if (tid == 0) {
            CHAIN_PROF(const long long tw = clock64(); hbusy += tw - hmark;)
            Spin sp;
            while (sh.ev_ready <= e && !sh.quit) {
                __nanosleep(32);
                if (sp.expired(2 * P.budget_ns + 1000000)) break;
            }
            CHAIN_PROF(hmark = clock64(); hidle += hmark - tw;)
            if (blockIdx.x == 1) P.out->dbg[7] = e;
            sh.hgo = sh.ev_ready > e;  // one decision for every compute thread
            __threadfence_block();     // the loader's column values before the barrier hands them on
        }
        cbar();
        if (!sh.hgo) { hflush(); return; }  // quit or abort
        const int s = e % NSLOT;
        const int kind = sh.ev[s].kind;
        const int np = sh.ev[s].np, a = sh.ev[s].a, b = sh.ev[s].b;
        const uint32_t W = sh.ev[s].s0;
        const uint32_t *za = sh.ring[s];
        const uint32_t *zb = sh.ring[s] + KP_MAX;
        if (kind == EV_END) {
            // rewrite this CTA's rows as true L columns
            const uint32_t *kinds = sh.ring[s];
            const uint32_t *cA = sh.ring[s] + KP_MAX;
            const uint32_t *cB = sh.ring[s] + 2 * KP_MAX;
            for (int k = tid; k < np; k += NCT) sh.kind[k] = (uint8_t)kinds[k];
            cbar();
            for (int lr = tid; lr < nrows; lr += NCT) {
                const int t = lo + lr;
                if (lr < SROWS) finish_row(P, sh.U + lr * RS, 1, P.LpC + t, np, sh.kind, cA, cB);
                else finish_row(P, P.LpT + t, (int)P.ldL, P.LpC + t, np, sh.kind, cA, cB);
            }
            hflush();
            return;
        }
        int firstnz = INT_MAX;
        for (int base = 0; base < nrows; base += NCT / 2) {
            const int lr = base + (tid >> 1);
            const bool valid = lr < nrows;
            const bool sm = lr < SROWS;
            const int t = lo + lr;
            const uint32_t sa = valid ? (sm ? sh.scol[s][0][lr] : s_at(P.S, P.ldS, t, a)) : 0u;
            if (kind == EV_PIVOT1) {
                const uint32_t c = schur2<BIG>(P, sh.U, lr, t, sa, W, za, np, half, valid, sm);
                if (valid && half == 0) {
                    if (sm) sh.U[lr * RS + np] = c;
                    else P.LpT[(int64_t)np * P.ldL + t] = c;
                }
            } else if (kind == EV_PIVOT2) {
                const uint32_t sb = valid ? (sm ? sh.scol[s][1][lr] : s_at(P.S, P.ldS, t, b)) : 0u;
                const uint32_t ca = schur2<BIG>(P, sh.U, lr, t, sa, W, za, np, half, valid, sm);
                const uint32_t cb = schur2<BIG>(P, sh.U, lr, t, sb, W, zb, np, half, valid, sm);
                if (valid && half == 0) {
                    if (sm) {
                        sh.U[lr * RS + np] = ca;
                        sh.U[lr * RS + np + 1] = cb;
                    } else {
                        P.LpT[(int64_t)np * P.ldL + t] = ca;
                        P.LpT[(int64_t)(np + 1) * P.ldL + t] = cb;
                    }
                }
            } else {  // EV_SCAN
                const uint32_t c = schur2<BIG>(P, sh.U, lr, t, sa, W, za, np, half, valid, sm);
                if (valid && c != 0 && t < firstnz) firstnz = t;
            }
        }
        if (kind == EV_SCAN && P.test_drop != 1) {
            for (int o = 16; o > 0; o >>= 1) firstnz = min(firstnz, __shfl_xor_sync(0xffffffffu, firstnz, o));
            if (lane == 0) sh.redi[warp] = firstnz;
            cbar();
            int mn = INT_MAX;
            for (int i = 0; i < NCW; ++i) mn = min(mn, sh.redi[i]);
            const int sid = sh.ev[s].scan_id;
            if (mn != INT_MAX) {
                // a hit: publish the candidate's columns, then the row index, then the count
                const int lr = mn - lo;
                uint32_t *dst = P.partner_lp +
                                ((int64_t)(sid % SCAN_RING) * MAX_PANEL_GRID + blockIdx.x) * PSTR;
                for (int k = tid; k < np; k += NCT)
                    dst[k] = lr < SROWS ? sh.U[lr * RS + k] : P.LpT[(int64_t)k * P.ldL + mn];
                __threadfence();
                cbar();
                if (tid == 0) {
                    atomicMin(&P.scans[sid].min, mn);
                    __threadfence();
                    atomicOr(&P.scans[sid].mask[blockIdx.x >> 5], 1u << (blockIdx.x & 31));
                    atomicAdd(&P.scans[sid].done, 1);
                }
            } else if (tid == 0) {
                // a miss: nothing to order before the answer bit and the count
                atomicOr(&P.scans[sid].mask[blockIdx.x >> 5], 1u << (blockIdx.x & 31));
                atomicAdd(&P.scans[sid].done, 1);
            }
        }
        cbar();
        if (tid == 0) { __threadfence_block(); sh.ev_done = e + 1; }
    }
}

// ---------------------------------------------------------------------------
// leader CTA
// ---------------------------------------------------------------------------
template <bool BIG>
__device__ void leader_cta(const PanelParams &P, Shared &sh, const int m, const int nh)
{
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const FieldP f = P.f;
    const int w = m < W0 ? m : W0;
    const bool helpers = nh > 0;
    for (int t = tid; t < W0; t += blockDim.x) sh.wstate[t] = 0;
    for (int i = tid; i < SRING; i += blockDim.x) sh.res_ok[i] = 0;
    for (int i = tid; i < SROWS * RS / 4; i += blockDim.x) reinterpret_cast<uint4 *>(sh.U)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        sh.np = 0; sh.ia = 0; sh.nzero = 0; sh.nscan = 0; sh.abort = 0; sh.nblk = 0;
        sh.ev_ready = 0; sh.ev_done = 0; sh.quit = 0; sh.W = 1u;
        sh.nscan_pub = 0; sh.ph_new = 0;
        sh.rb = -1; sh.nrollback = 0;
        for (int i = 0; i < 16; ++i) sh.dbg[i] = 0;
    }
    __syncthreads();

    if (warp == NCW + 1) {
        // ---- publisher: every ready ring slot -> global, one fence, then the counter ----
        if (!helpers) return;
        int e = 0;
        int last_scan = -1;
        for (;;) {
            int ready = 0;
            if (lane == 0) {
                Spin sp;
                for (;;) {
                    const int r = sh.ev_ready;
                    if (r > e) { ready = r; break; }
                    if (sh.quit) break;
                    __nanosleep(20);
                    if (sp.expired(4 * P.budget_ns + 1000000)) break;
                }
            }
            ready = __shfl_sync(0xffffffffu, ready, 0);
            if (!ready) return;
            __threadfence_block();
            bool end = false;
            for (int ee = e; ee < ready; ++ee) {
                const int s = ee % NSLOT;
                const int kind = sh.ev[s].kind, np = sh.ev[s].np;
                uint32_t *rec = P.evlog + (int64_t)ee * EV_REC;
                const int words = (kind == EV_END) ? 3 * KP_MAX : (kind == EV_PIVOT2 ? 2 * KP_MAX : KP_MAX);
                for (int k = lane; k < words; k += 32) {
                    const int kk = k % KP_MAX;
                    // z vectors with their zero padding to a multiple of 8
                    if (kind == EV_END || kk < ((np + 7) & ~7)) rec[8 + k] = sh.ring[s][k];
                }
                if (lane < 8) rec[lane] = reinterpret_cast<const uint32_t *>(&sh.ev[s])[lane];
                if (kind == EV_SCAN) {
                    const int sid = sh.ev[s].scan_id;
                    if (lane < 8) P.scans[sid].mask[lane] = 0u;
                    if (lane == 0) {
                        P.scans[sid].done = 0;
                        P.scans[sid].min = INT_MAX;
                    }
                    last_scan = sid;
                }
                end = end || (kind == EV_END);
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                atomicExch(&P.sync->ev_count, ready);
                sh.dbg[8] += 1;
                sh.dbg[9] += ready - e;
                sh.ev_done = ready;
                if (last_scan >= 0) sh.nscan_pub = last_scan + 1;  // the watcher may poll those slots now
            }
            __syncwarp();
            if (end) return;
            e = ready;
        }
    }
    if (warp == NCW) {
        // ---- watcher: posts the answers of the far scans ----
        // Lane i probes scan base + i, so up to 32 published scans are watched
        // at once and each answer is posted as soon as it is final: a miss
        // once every helper answered; a hit at row v once the helpers owning
        // the rows below v answered (no smaller row can still come), which
        // is usually well before the last helper is done.
        if (!helpers) return;
        const int chunk = (m - w + nh - 1) / nh;  // far rows per helper, as in helper_cta
        volatile int *ab = &P.sync->abort;
        int base = 0;
        unsigned posted = 0u;  // bit i: scan base + i posted
        Spin sp;
        for (;;) {
            const int npub = sh.nscan_pub;
            const int id = base + lane;
            bool ok = false;
            if (id < npub && !((posted >> lane) & 1u)) {
                const ScanSlot *sl = P.scans + id;
                int v = INT_MAX;
                if (ld_acquire(&sl->done) >= nh) {
                    v = __ldcg(&sl->min);
                    ok = true;
                } else {
                    const int m = (int)ld_relaxed(&sl->min);
                    if (m != INT_MAX) {
                        const int owner = 1 + (m - w) / chunk;
                        bool all = true;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            if (32 * i > owner) break;
                            const int b0 = 32 * i < 1 ? 1 : 32 * i;
                            const int b1 = 32 * i + 31 < owner ? 32 * i + 31 : owner;
                            const unsigned need = (b1 - 32 * i == 31 ? 0xffffffffu : ((2u << (b1 - 32 * i)) - 1u)) &
                                                  ~((1u << (b0 - 32 * i)) - 1u);
                            const unsigned got = ld_relaxed(&sl->mask[i]);
                            all = all && ((got & need) == need);
                        }
                        if (all) {
                            // every helper below owner answered; acquire their
                            // mins, then the smallest row is final
                            asm volatile("fence.acq_rel.gpu;" ::: "memory");
                            v = (int)ld_relaxed(&sl->min);
                            ok = true;
                        }
                    }
                }
                if (ok) {
                    sh.res_min[id % SRING] = v;
                    __threadfence_block();
                    sh.res_ok[id % SRING] = id + 1;
                }
            }
            const unsigned okm = __ballot_sync(0xffffffffu, ok);
            posted |= okm;
            const int adv = (posted == 0xffffffffu) ? 32 : __ffs(~posted) - 1;
            base += adv;
            posted = (adv == 32) ? 0u : (posted >> adv);
            if (okm) {
                sp = Spin();
                continue;
            }
            if (sh.quit) return;
            // lane 0 decides for the warp when to give up
            int stop = 0;
            if (lane == 0) {
                if (base < npub) {
                    if (*ab) stop = 1;
                    else if (sp.expired(P.budget_ns)) { raise_timeout(P); stop = 1; }
                } else {
                    __nanosleep(32);
                    if (sp.expired(4 * P.budget_ns + 1000000)) stop = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) return;
        }
    }

    // ---- compute warps: 512 threads, two per window row ----
    // The control state lives in registers, identical in every compute
    // thread: each update is computed from values every thread reads after
    // a barrier, so the threads never diverge on it.
    const int half = tid & 1;
    const int lr = tid >> 1;  // window row of this thread pair
    const bool inwin = lr < w;
    int np = 0, ia = 0, nzero = 0, nscan = 0, ph = 0, pt = 0, ev_next = 0, nrb = 0;
    int force_b = -1, force_sid = -1;
    uint32_t W = 1u;
    // S[lr][4g .. 4g+3] of this thread's window row for the current column
    // group g = a / 4 and the next one: one 16-byte load per four rows, issued
    // a group ahead, keeps the DRAM latency off the per-row chain
    uint4 g_cur = make_uint4(0, 0, 0, 0), g_nxt = make_uint4(0, 0, 0, 0);
    int cur_g = -1, nxt_g = -1;
    auto load_grp = [&](int g) -> uint4 {
        if (inwin && lr >= 4 * g) return __ldg(reinterpret_cast<const uint4 *>(P.S + (int64_t)lr * P.ldS + 4 * g));
        return make_uint4(0, 0, 0, 0);
    };

    // ring slot e % NSLOT may be written once event e - NSLOT is published
    auto ring_ready = [&](int e) {
        if (sh.ev_done <= e - NSLOT) {
            Spin sp;
            while (sh.ev_done <= e - NSLOT) {
                __nanosleep(16);
                if (sp.expired(P.budget_ns)) { raise_timeout(P); sh.abort = 1; break; }
            }
        }
    };
    // the control warp (lane 0 is CTL): take in the answered scans.  Posts
    // the new head (the first pending scan that is unanswered or found a
    // partner) and a rollback request: the earliest answered scan that found a
    // partner (-1 if none), even while older scans are still unanswered; they
    // stay pending and may roll the panel back further.
    auto resolved = [&](int id) { return ld_acquire_cta(&sh.res_ok[id % SRING]) == id + 1; };
    auto check_scans = [&](bool wait_oldest) {
        __syncwarp();  // the pend_* records written by CTL
        if (wait_oldest && ph < pt) {
            if (lane == 0) {
                const int id = sh.pend_id[ph % NPEND];
                Spin sp;
                while (!resolved(id)) {
                    __nanosleep(16);
                    if (sp.expired(P.budget_ns)) { raise_timeout(P); sh.abort = 1; break; }
                }
                sh.dbg[1] += 1;
            }
            __syncwarp();
        }
        const int q = ph + lane;  // pt - ph <= NPEND < 32
        bool res = false, hit = false;
        int v = 0;
        if (q < pt) {
            const int id = sh.pend_id[q % NPEND];
            if (resolved(id)) {  // the answer is read only after its flag
                res = true;
                v = sh.res_min[id % SRING];
                hit = v >= w && v < m;
            }
        }
        const unsigned rm = __ballot_sync(0xffffffffu, res), hm = __ballot_sync(0xffffffffu, hit);
        const int head = __ffs(~rm | hm) - 1;
        const int first = hm ? __ffs(hm) - 1 : -1;
        const int vb = __shfl_sync(0xffffffffu, v, first < 0 ? 0 : first);
        if (lane == 0) {
            sh.ph_new = ph + head;
            sh.rb = first < 0 ? -1 : ph + first;
            sh.rb_b = vb;
        }
    };
    // all compute threads: roll back to pending scan k, which found partner b
    auto rollback = [&](int k, int bfound) {
        const int slot = k % NPEND;
        const int ak = sh.pend_row[slot], npk = sh.pend_np[slot];
        for (int j = npk + tid; j < np; j += NCT)
            if (sh.kind[j] == K_2B) P.consumed[sh.piv_rows[j]] = 0;
        for (int t = ak + tid; t < w; t += NCT) sh.wstate[t] = 0;
        cbar();
        for (int j = tid; j < npk; j += NCT) {
            if (sh.kind[j] == K_2B) {
                const int bb = sh.piv_rows[j];
                if (bb >= ak && bb < w) sh.wstate[bb] = 1;
            }
            sh.bw[j] = sh.pend_bw[slot][j];
        }
        for (int q = tid; q < (np - npk) * w; q += NCT) {
            const int j = npk + q / w, t = q % w;
            sh.U[t * RS + j] = 0;
        }
        np = npk;
        nzero = sh.pend_nz[slot];
        ia = ak;
        W = sh.pend_W[slot];
        force_b = bfound;
        force_sid = sh.pend_id[slot];
        pt = k;  // this and every later pending scan are dropped; older ones stay
        ++nrb;
        cbar();
    };

    long long cyc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    CHAIN_PROF(long long tmark = clock64();)
    auto lap = [&](int phz) {
        CHAIN_PROF(if (tid == 0) { const long long t = clock64(); cyc[phz] += t - tmark; tmark = t; })
        (void)phz;
    };

    for (;;) {
        const bool full = np > P.kp - 2 || ia >= w || ev_next > MAX_EVENTS - 64 || nscan > MAX_SCANS - 64;
        if (full) {
            if (ph == pt) break;  // nothing in flight: the panel is complete
            if (warp == NCW - 1) check_scans(true);
            cbar();
            ph = sh.ph_new;
            const int rb = sh.rb, rb_b = sh.rb_b;
            const bool ab = sh.abort;
            cbar();
            if (ab) break;
            if (rb >= 0) rollback(rb, rb_b);
            lap(6);
            continue;
        }
        if (sh.wstate[ia]) {
            ++ia;
            continue;
        }
        const int a = ia;
        const int slot = ev_next % NSLOT;
        uint32_t *za = sh.ring[slot];
        uint32_t *zb = sh.ring[slot] + KP_MAX;
        // z beyond np up to the next multiple of 8 is zero: the dot products read
        // whole 8-column groups and a CTA's U~ may hold stale columns there
        // (written before a rollback)
        if (tid < ((np + 7) & ~7)) {
            ring_ready(ev_next);
            za[tid] = tid < np ? zval(tid, sh.U + a * RS, 1, sh, f) : 0u;
        }
        if (warp == NCW - 1) {
            if (lane == 0) sh.dbg[0] += 1;
            check_scans(false);
        }
        const bool myrow = inwin && lr >= a;
        {
            const int g = a >> 2;
            if (g != cur_g) {
                g_cur = (nxt_g == g) ? g_nxt : load_grp(g);
                cur_g = g;
                if (4 * (g + 1) < w) g_nxt = load_grp(g + 1);
                nxt_g = g + 1;
            }
        }
        const uint32_t s_col = myrow ? pick4(g_cur, a & 3) : 0u;
        CHAIN_PROF(const long long tb1 = clock64();)
        cbar();
        CHAIN_PROF(const long long ta1 = clock64();)
        {
            ph = sh.ph_new;
            const int rb = sh.rb, rb_b = sh.rb_b;
            if (sh.abort) break;
            if (rb >= 0) {
                cbar();  // every thread has read the posted request
                rollback(rb, rb_b);
                lap(5);
                continue;
            }
        }
        // Snapshot for a rollback to this row, kept if its scan is issued.  It
        // is taken after the head update above, with the head the scan path
        // tests: a scan goes out only while pt - ph < npend <= NPEND, so slot
        // pt % NPEND then holds no pending scan's snapshot and always holds
        // this row's.
        if (tid < np && pt - ph < NPEND) sh.pend_bw[pt % NPEND][tid] = sh.bw[tid];
        lap(0);
        // c~_a[t] for the window rows t >= a (t = a included) and the first
        // non-zero of row a beyond a inside the window, in one pass
        const uint32_t ca_t = schur2<BIG>(P, sh.U, lr, lr, s_col, W, za, np, half, myrow, true);
        if (lr == a && half == 0) sh.caa = ca_t;
        int firstnz = (half == 0 && inwin && lr > a && ca_t != 0) ? lr : INT_MAX;
        for (int o = 16; o > 0; o >>= 1) firstnz = min(firstnz, __shfl_xor_sync(0xffffffffu, firstnz, o));
        if (lane == 0) sh.redi[warp] = firstnz;
        CHAIN_PROF(const long long tb2 = clock64();)
        cbar();
        CHAIN_PROF(const long long ta2 = clock64();)
        CHAIN_PROF(if (tid == 0 || tid == NCT - 1) {
            const int o = (tid == 0) ? 10 : 12;
            sh.dbg[o] += ta1 - tb1;       // wait at barrier 1
            sh.dbg[o + 1] += ta2 - tb2;   // wait at barrier 2
            if (tid == 0) sh.dbg[14] += tb2 - ta1;  // schur phase (thread 0)
            else sh.dbg[15] += tb2 - ta1;
        })
        lap(1);
        const uint32_t caa = sh.caa;

        if (caa != 0) {
            // ---- 1x1 pivot: U~[:, np] = c~_a, delta = W c~_a[a] ----
            if (myrow && half == 0) {
                sh.U[lr * RS + np] = ca_t;
            }
            const uint32_t delta = fp_mul(W, caa, f);
            if (tid < np && sh.kind[tid] != K_2B) sh.bw[tid] = fp_mul(sh.bw[tid], delta, f);
            if (tid == 0) {
                if (helpers) {
                    Event &ev = sh.ev[slot];
                    ev.kind = EV_PIVOT1; ev.a = a; ev.b = -1; ev.np = np; ev.s0 = W; ev.col = np;
                    ev.scan_id = 0; ev.aux = 0;
                    __threadfence_block();
                    sh.ev_ready = ev_next + 1;
                }
                sh.kind[np] = K_1x1; sh.bw[np] = W; sh.piv[np] = caa; sh.w0[np] = W; sh.delta[np] = delta;
                sh.piv_rows[np] = a;
                sh.wstate[a] = 1;
            }
            W = fp_mul(W, delta, f);
            ++np;
            ++ia;
            if (helpers) ++ev_next;
            cbar();
            lap(2);
            continue;
        }

        int b = INT_MAX;
        bool far = false;
        if (force_b >= 0) {
            // partner found by this row's scan before the rollback
            b = force_b;
            far = true;
            const int chunk = (m - w + nh - 1) / nh;
            const int owner = 1 + (b - w) / chunk;
            const uint32_t *src = P.partner_lp +
                                  ((int64_t)(force_sid % SCAN_RING) * MAX_PANEL_GRID + owner) * PSTR;
            if (tid < np) sh.ub[tid] = __ldcg(src + tid);
        } else {
            for (int i = 0; i < NCW; ++i) b = min(b, sh.redi[i]);
        }
        if (b == INT_MAX && helpers) {
            // ---- speculative far scan: publish it and go on as if the row were zero ----
            if (pt - ph >= P.npend) {
                if (warp == NCW - 1) check_scans(true);
                cbar();
                ph = sh.ph_new;
                const int rb = sh.rb, rb_b = sh.rb_b;
                const bool ab = sh.abort;
                cbar();
                if (ab) break;
                if (rb >= 0) rollback(rb, rb_b);
                lap(6);
                continue;  // the row is taken again from the top
            }
            if (tid == CTL) {
                Event &ev = sh.ev[slot];
                ev.kind = EV_SCAN; ev.a = a; ev.b = -1; ev.np = np; ev.s0 = W; ev.col = -1;
                ev.scan_id = nscan; ev.aux = 0;
                const int ps = pt % NPEND;
                sh.pend_id[ps] = nscan; sh.pend_row[ps] = a; sh.pend_np[ps] = np;
                sh.pend_nz[ps] = nzero; sh.pend_W[ps] = W;
                sh.zero_rows[nzero] = a; sh.zero_np[nzero] = np;
                sh.wstate[a] = 1;
                __threadfence_block();
                sh.ev_ready = ev_next + 1;
            }
            ++nscan;
            ++pt;
            ++nzero;
            ++ia;
            ++ev_next;
            lap(3);
            continue;
        }
        if (b == INT_MAX) {
            // ---- zero row (no far rows to search) ----
            if (tid == 0) {
                sh.zero_rows[nzero] = a; sh.zero_np[nzero] = np;
                sh.wstate[a] = 1;
            }
            ++nzero;
            ++ia;
            continue;
        }

        // ---- 2x2 pivot on (a, b) ----
        // S(a, b) and S(b, b) for x~ and y~, loaded before the z work below
        uint32_t s_ab = 0u, s_bb = 0u;
        if (tid == 0) {
            s_ab = s_at(P.S, P.ldS, a, b);
            s_bb = s_at(P.S, P.ldS, b, b);
        }
        if (!far && tid < np) sh.ub[tid] = sh.U[b * RS + tid];
        cbar();
        if (tid < ((np + 7) & ~7)) zb[tid] = tid < np ? zval(tid, sh.ub, 1, sh, f) : 0u;
        cbar();
        // x~ = W S(a,b) - U~[b] . z_a ;  y~ = W S(b,b) - U~[b] . z_b   (warp 0)
        if (warp == 0) {
            uint64_t ax = 0, ay = 0;
            for (int k = lane; k < np; k += 32) {
                mac<true>(ax, sh.ub[k], za[k], f);
                mac<true>(ay, sh.ub[k], zb[k], f);
            }
            uint64_t sx = fp_reduce64(ax, f), sy = fp_reduce64(ay, f);
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane == 0) {
                sh.xy[0] = fp_sub(fp_mul(W, s_ab, f), fp_reduce64(sx, f), f);
                sh.xy[1] = fp_sub(fp_mul(W, s_bb, f), fp_reduce64(sy, f), f);
            }
        }
        // c~_b[t] for the window rows t >= a (overlaps warp 0's work)
        const uint32_t s_b = myrow ? s_at(P.S, P.ldS, lr, b) : 0u;
        const uint32_t cb_t = schur2<BIG>(P, sh.U, lr, lr, s_b, W, zb, np, half, myrow, true);
        cbar();
        const uint32_t x = sh.xy[0], y = sh.xy[1];
        if (myrow && half == 0) {
            sh.U[lr * RS + np] = ca_t;  // c~_a[a] = 0 here
            sh.U[lr * RS + np + 1] = cb_t;
        }
        const uint32_t delta = fp_mul(W, fp_mul(x, x, f), f);
        if (tid < np && sh.kind[tid] != K_2B) sh.bw[tid] = fp_mul(sh.bw[tid], delta, f);
        if (tid == 0) {
            if (helpers) {
                Event &ev = sh.ev[slot];
                ev.kind = EV_PIVOT2; ev.a = a; ev.b = b; ev.np = np; ev.s0 = W; ev.col = np;
                ev.scan_id = 0; ev.aux = 0;
                __threadfence_block();
                sh.ev_ready = ev_next + 1;
            }
            sh.kind[np] = K_2A; sh.kind[np + 1] = K_2B;
            sh.bw[np] = W; sh.mx[np] = x; sh.my[np] = y; sh.piv[np] = x; sh.w0[np] = W;
            sh.delta[np] = delta;
            sh.piv_rows[np] = a; sh.piv_rows[np + 1] = b;
            sh.wstate[a] = 1;
            if (b < w) sh.wstate[b] = 1;
            P.consumed[b] = 1;
        }
        W = fp_mul(W, delta, f);
        np += 2;
        ++ia;
        if (helpers) ++ev_next;
        force_b = -1;
        force_sid = -1;
        cbar();
        lap(4);
    }
    if (tid == 0) {
        sh.np = np; sh.ia = ia; sh.nzero = nzero; sh.nscan = nscan; sh.nrollback = nrb;
    }
    cbar();

    // ---- end of panel: batch inversion, true D and the L coefficients ----
    const int iend = ia;
    if (!sh.abort) {
        if (tid == 0) {
            // per block: its pivot value and its W, inverted together (Montgomery's trick)
            int nv = 0;
            for (int j = 0; j < np; ++j)
                if (sh.kind[j] != K_2B) { sh.bi[nv++] = sh.piv[j]; sh.bi[nv++] = sh.w0[j]; }
            uint32_t run = 1;
            for (int i = 0; i < nv; ++i) { run = fp_mul(run, sh.bi[i], f); sh.bpre[i] = run; }
            uint32_t inv = nv ? fp_inv_bin(run, f) : 1u;
            for (int i = nv - 1; i >= 0; --i) {
                const uint32_t before = i ? sh.bpre[i - 1] : 1u;
                const uint32_t vi = sh.bi[i];
                sh.bi[i] = fp_mul(inv, before, f);  // inverse of value i
                inv = fp_mul(inv, vi, f);
            }
            int v = 0;
            for (int j = 0; j < np; ++j) {
                const uint8_t kd = sh.kind[j];
                if (kd == K_1x1) {
                    const uint32_t ipiv = sh.bi[v], iw0 = sh.bi[v + 1];
                    v += 2;
                    sh.cA[j] = ipiv;
                    sh.cB[j] = 0;
                    sh.dtrue[j] = fp_mul(sh.piv[j], iw0, f);
                    sh.etrue[j] = 0;
                } else if (kd == K_2A) {
                    const uint32_t ix = sh.bi[v], iw0 = sh.bi[v + 1];
                    v += 2;
                    const uint32_t yt = sh.my[j];
                    const uint32_t dl = (f.p == 2) ? yt : fp_mul(yt, f.inv2, f);
                    sh.cA[j] = ix;
                    sh.cB[j] = fp_sub(0, fp_mul(dl, fp_mul(ix, ix, f), f), f);
                    sh.cA[j + 1] = ix;
                    sh.cB[j + 1] = 0;
                    sh.dtrue[j] = 0;
                    sh.dtrue[j + 1] = (f.p == 2) ? fp_mul(yt, iw0, f) : 0u;
                    sh.etrue[j] = fp_mul(sh.mx[j], iw0, f);
                    sh.etrue[j + 1] = 0;
                    ++j;
                }
            }
        }
        cbar();
        if (helpers) {
            for (int k = tid; k < np; k += NCT) sh.bpre[k] = sh.kind[k];
            cbar();
            // the end event carries the column kinds and the true-L coefficients
            const int slot = ev_next % NSLOT;
            if (tid < np) {
                ring_ready(ev_next);
                sh.ring[slot][tid] = sh.bpre[tid];
                sh.ring[slot][KP_MAX + tid] = sh.cA[tid];
                sh.ring[slot][2 * KP_MAX + tid] = sh.cB[tid];
            }
            if (tid == 0) ring_ready(ev_next);
            cbar();
            if (tid == 0) {
                Event &ev = sh.ev[slot];
                ev.kind = EV_END; ev.a = -1; ev.b = -1; ev.np = np; ev.s0 = 0; ev.col = np;
                ev.scan_id = 0; ev.aux = 0;
                __threadfence_block();
                sh.ev_ready = ev_next + 1;
            }
        }
        // rewrite the window rows as true L columns
        for (int t = tid; t < w; t += NCT) finish_row(P, sh.U + t * RS, 1, P.LpC + t, np, sh.kind, sh.cA, sh.cB);
    }
    cbar();
    if (tid == 0) { __threadfence_block(); sh.quit = 1; }
    __threadfence();
    cbar();

    // ---- report: D and x for the update, the pivots and zero rows (as
    // original indices) appended to the factorisation's lists ----
    {
        const int r0 = P.ls->r0, z0 = P.ls->z0;
        for (int k = tid; k < np; k += NCT) {
            P.out->dval[k] = sh.dtrue[k];
            P.out->eval[k] = sh.etrue[k];
            P.piv_all[r0 + k] = P.idx[sh.piv_rows[k]];
            P.d_all[r0 + k] = sh.dtrue[k];
            P.e_all[r0 + k] = sh.etrue[k];
        }
        for (int q = tid; q < nzero; q += NCT) {
            P.zero_all[z0 + q] = P.idx[sh.zero_rows[q]];
            P.zero_cols[z0 + q] = r0 + sh.zero_np[q];  // L columns that existed when it was found zero
        }
    }

    // ---- compaction of the remaining rows [iend, m) minus consumed partners ----
    const int len = m - iend;
    const int per = (len + NCT - 1) / NCT;
    const int lo = iend + tid * per, hi = min(m, lo + per);
    int cnt = 0;
    for (int t = lo; t < hi; ++t) cnt += P.consumed[t] ? 0 : 1;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int vv = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += vv;
    }
    if (lane == 31) sh.redi[warp] = incl;
    cbar();
    int woff = 0, total = 0;
    for (int i = 0; i < NCW; ++i) {
        if (i < warp) woff += sh.redi[i];
        total += sh.redi[i];
    }
    int pos = woff + incl - cnt;
    for (int t = lo; t < hi; ++t) {
        if (!P.consumed[t]) {
            P.sigma[pos] = t;
            P.idx_next[pos] = P.idx[t];
            ++pos;
        }
    }
    if (tid == 0) {
        P.out->np = np;
        P.out->nzero = nzero;
        P.out->iend = iend;
        P.out->m_next = total;
        P.out->abort = sh.abort | *((volatile int *)&P.sync->abort);
        P.out->nscan = sh.nscan;
        P.out->pad[0] = sh.nrollback;
        for (int i = 0; i < 8; ++i) P.out->cyc[i] = cyc[i];
        sh.dbg[4] = sh.nrollback;
        for (int i = 0; i < 16; ++i)
            if (i < 5 || i > 7) P.out->dbg[i] = sh.dbg[i];
    }
}

template <bool BIG>
__global__ void __launch_bounds__(BLOCK, 1) panel_kernel(PanelParams P)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    Shared &sh = *reinterpret_cast<Shared *>(smem_raw);
    // the loop state was written by earlier kernels: every CTA reads the same
    if (P.ls->done) return;
    const int m = P.ls->m;
    const int ncta = panel_grid(m, gridDim.x);  // the grid is sized for the first panel
    if (blockIdx.x >= ncta) return;
    if (*(volatile int32_t *)P.status != 0) {
        // an earlier kernel of this factorisation gave up: end it here
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            P.out->np = 0; P.out->nzero = 0; P.out->iend = 0; P.out->m_next = 0;
            P.out->abort = 1; P.out->nscan = 0;
        }
        return;
    }
    const int nh = ncta - 1;
    if (blockIdx.x == 0) {
        leader_cta<BIG>(P, sh, m, nh);
    } else {
        const int w = m < W0 ? m : W0;
        const int chunk = (m - w + nh - 1) / nh;
        const int lo = w + (blockIdx.x - 1) * chunk;
        const int hi = min(m, lo + chunk);
        helper_cta<BIG>(P, sh, lo, hi);
    }
}

}  // namespace

cudaError_t launch_panel(const PanelParams &pp, int grid, cudaStream_t st)
{
    PanelParams p = pp;
    void *args[] = {&p};
    const bool big = pp.f.p >= (1u << 28);
    const void *fn = big ? (const void *)panel_kernel<true> : (const void *)panel_kernel<false>;
    const size_t smem = sizeof(Shared);
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    if (grid <= 1) return cudaLaunchKernel(fn, dim3(1), dim3(BLOCK), args, smem, st);
    // the CTAs wait on one another: all of them must be resident at once
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BLOCK);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}
