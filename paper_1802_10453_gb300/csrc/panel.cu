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
// With a common scale W and weights w_B = W / delta_B (kept by multiplication
// only for the blocks the window decides) the scaled Schur entry is
//   c~_a[t] = W c_a[t] = W S[t][a] - sum_k U~[t][k] z_a[k],
//   z_a = concat_B  M_B U~[a][B]^T w_B,
// and c~ is zero exactly when c is.  A 1x1 pivot stores U~[:, j] = c~_a
// (M = 1, delta = W c~_a[a]); a 2x2 pivot stores c~_a and c~_b
// (M = [[-y~, x~], [x~, 0]], delta = W x~^2, x~ = c~_a[b], y~ = c~_b[b]).  The
// block forms follow from Algorithm 4's 2x2 branch: with beta = c_a / x,
// alpha = (c_b - delta' beta) / x and D = [[0,x],[x,y']], the product
// [alpha, beta] D [alpha', beta']^T equals [c_a, c_b] [[-y/x^2, 1/x],[1/x, 0]]
// [c_a', c_b']^T for both odd p (y' = 0, delta' = y/2) and p = 2 (y' = delta'
// = y).  Each block keeps the scale W it was formed with (its columns, pivot
// and delta all carry it), so blocks need not share one scale.  At the end of
// the panel all inverses are taken at once (Montgomery's batch inversion) and
// every CTA rewrites its rows as the true L columns, in pivot order; D is
// reported in true values.  All arithmetic is exact, so the results equal the
// divided form bit for bit.
//
// Far pairs without rollback.  A window row whose Schur row is zero inside the
// window is a zero row or the first row a of a 2x2 pivot (a, b) with a far
// partner b.  The helpers search the far part of the row (a "far scan") while
// the leader goes on as if the row were zero.  When the scan finds b, the
// block (a, b) belongs before every block the leader took since row a, but it
// changes none of their window values: c_a[t] = 0 for every window row t > a,
// so the block's share of c_u[t], proportional to c_a[t] c_b[u] + c_b[t] c_a[u],
// vanishes when t and u are both window rows.  So every window decision stands
// and the leader only
//   * forms the block's window column c~_b (one pass with row b's values at
//     the scan's position) and its weight W / delta from one true inverse, so
//     that W keeps counting window blocks only;
//   * tells the helpers, whose far columns of the later blocks lack the
//     block's share.  By linearity each such column needs a rank-1 fix,
//     new = old - c~_a[t] rho, where c~_a is the scan's own column (kept by the
//     helpers) and rho a scalar per column that the leader computes by a short
//     triangular recurrence over the later blocks.  The later scans' columns
//     get the same fix and are answered again under new ids.
// Scans are settled in order, so a block is inserted only when every scan
// before it found no partner.
//
// GPU organisation.  One cooperative launch per panel.  CTA 0 (the leader)
// owns the window of the first W rows of S and takes every decision.  The
// other CTAs (helpers) own the far rows [W, m) in contiguous slices.  Each CTA
// keeps the U~ columns of its rows in shared memory (k-major, padded) and
// writes them through to global memory.  16 compute warps work two threads
// per row.  In the leader, warp 17 publishes events to the helpers from a
// shared-memory ring so the gpu-scope fence stays off the critical path, and
// warp 16 watches the scan answers; in a helper, warp 16 fetches events into
// the ring and warp 17 loads the Schur columns they need.  Every wait is
// bounded by a %globaltimer budget; when it runs out the kernel writes
// LDLT_ERR_TIMEOUT to the status word, raises an abort flag the other CTAs
// poll, and returns.
//
// At the end the leader compacts the remaining rows (order preserved) into
// sigma / idx_next for the next Schur complement.
#include <climits>

#include "ldlt_internal.cuh"

#define LDLT_ERR_TIMEOUT_CODE (-6)

namespace {

constexpr int NCW = 16;                       // compute warps
constexpr int NCT = NCW * 32;                 // compute threads (2 per row)
constexpr int SROWS = 256;                    // rows held in shared memory per CTA
constexpr int SSTRIDE = SROWS + 16;           // padded k-row stride (words)
constexpr int NSLOT = 8;                      // event ring slots
constexpr int BLOCK = PANEL_THREADS_V2;
constexpr int NPEND = 16;                     // far scans in flight
constexpr int EVT = 64;                       // leader's table of recent row events (ring)
constexpr int EVT_LIM = 40;                   // row events since the oldest pending scan
constexpr int LPL = 3;                        // corrected columns per lane (3 * 32 >= 2 * EVT_LIM)
constexpr int SRING = 128;                    // posted scan results

static_assert(BLOCK == NCT + 64, "two service warps");
static_assert(W0 <= SROWS && ROWS_PER_HELPER <= SROWS, "rows fit in shared memory");
static_assert(W0 <= NCT / 2, "one thread pair per window row");
static_assert(LPL * 32 >= 2 * EVT_LIM, "corrected columns fit the sweep's lanes");
static_assert(KP_MAX + 2 * (2 * EVT_LIM) + 3 * NPEND <= EV_WORDS, "far-pair payload fits an event");
static_assert(2 * NPEND + 8 < SCAN_RING && 2 * NPEND + 8 < SRING, "scan id rings");

enum ColKind : uint8_t { K_1x1 = 1, K_2A = 2, K_2B = 3 };
// window row states (leader)
constexpr int RI_UNDEC = 0, RI_PART = 1, RI_ZERO = 2, RI_PEND = 3, RI_PIV = 4;  // RI_PIV + storage column
constexpr int EK_P1 = 1, EK_P2 = 2, EK_SCAN = 3;                                 // row-event kinds

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

struct Shared {
    uint32_t U[KP_MAX * SSTRIDE];      // U~ columns of this CTA's rows, k-major
    uint32_t ring[NSLOT][EV_WORDS];    // event payloads
    uint32_t scol[NSLOT][2][SROWS];    // helpers: S(t, a) and S(t, b) of each ring event
    uint4 sgrp[2][SROWS];              // helpers: S[t][4g .. 4g+3] for two column groups
    Event ev[NSLOT];
    uint32_t ub[KP_MAX];               // U~ row of a 2x2 partner
    uint32_t zt[KP_MAX];               // z vector of a far partner
    uint8_t kind[KP_MAX];              // column kinds (storage order); far pairs are K_2A / K_2B
    uint8_t isfar[KP_MAX];             // 1 on both columns of a far pair
    uint32_t bw[KP_MAX];               // weight W / delta_B, at the block's first column
    uint32_t mx[KP_MAX], my[KP_MAX];   // x~, y~ of a 2x2 block (first column)
    uint32_t piv[KP_MAX];              // c~_a[a] (1x1) or x~ (2x2) at the first column
    uint32_t w0[KP_MAX];               // the block's own scale W
    uint32_t delta[KP_MAX];            // delta_B (window blocks) at the first column
    uint32_t invd[KP_MAX];             // 1 / delta_B (far pairs) at the first column
    int brow[KP_MAX];                  // window row of the block, at both columns
    uint32_t cA[KP_MAX], cB[KP_MAX];   // true-L coefficients (end of panel)
    uint32_t dtrue[KP_MAX], etrue[KP_MAX];
    uint32_t bi[2 * KP_MAX];           // batch inversion: values, then their inverses
    uint32_t bpre[2 * KP_MAX];         // batch inversion: prefix products
    int piv_rows[KP_MAX];              // compact rows, storage order
    int canon[KP_MAX];                 // storage column -> pivot-order position
    int rinfo[W0];                     // window row state RI_*
    // far scans in flight (FIFO, settled from the head)
    int pend_id[NPEND], pend_row[NPEND], pend_ev[NPEND];
    uint32_t pend_W[NPEND];
    uint32_t pend_bw[NPEND][KP_MAX];   // block weights when the scan was issued
    // table of recent row events (absolute index mod EVT)
    int evt_kind[EVT], evt_u[EVT], evt_v[EVT], evt_col[EVT], evt_sid[EVT];
    uint32_t evt_W[EVT];
    int res_min[SRING];
    volatile int res_ok[SRING];        // id + 1 once scan id's answer is in res_min
    int redi[32];
    int redj[32];
    uint32_t xy[4];
    uint32_t caa;
    volatile int ev_ready;             // events written to the ring (leader) / fetched (helper)
    volatile int ev_done;              // events published (leader) / processed (helper)
    volatile int quit;
    volatile int ev_fetched;           // helpers: event records fetched (poller -> column loader)
    volatile int nscan_pub;            // scans published (leader -> watcher warp)
    int head_new, head_b;              // posted by the control warp: settled head, hit partner
    int ncorr, nres;                   // far pair: corrections and re-issued scans in its event
    int hgo;                           // helpers: the next event is in the ring (tid 0's decision)
    int abort;
    long long dbg[16];                 // counters (thread-0 owned)
};

// load with acquire semantics at GPU scope
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

// acquire load at CTA scope, for flags in shared memory
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

// z[k] of row u (u read with a stride) with the block weight wt:
// M_B U~[u][B]^T w_B for the block holding column k.
__device__ __forceinline__ uint32_t zval_w(int k, const uint32_t *u, int stride, const Shared &sh, uint32_t wt,
                                           const FieldP &f)
{
    const uint8_t kd = sh.kind[k];
    const int kb = k - (kd == K_2B);               // the block's first column
    const int j = k + (kd == K_2A) - (kd == K_2B);
    const uint32_t c1 = kd == K_1x1 ? 1u : sh.mx[kb];
    const uint32_t c2 = kd == K_2A ? sh.my[k] : 0u;
    const uint32_t t = fp_sub(fp_mul(c1, u[j * stride], f), fp_mul(c2, u[k * stride], f), f);
    return fp_mul(t, wt, f);
}

__device__ __forceinline__ uint32_t zval(int k, const uint32_t *u, int stride, const Shared &sh, const FieldP &f)
{
    return zval_w(k, u, stride, sh, sh.bw[k - (sh.kind[k] == K_2B)], f);
}

// c~_z[t] = W S(t, a) - sum_{k < np} U~[t][k] z[k], two threads per row (half
// = tid & 1 takes every other k).  All 32 lanes must call it (pair shuffle);
// invalid rows compute nothing and return 0.
template <bool BIG>
__device__ __forceinline__ uint32_t schur2(const PanelParams &P, const uint32_t *sU, int lrow, int grow,
                                          uint32_t sval, uint32_t W, const uint32_t *z, int np, int half,
                                          bool valid, bool in_smem)
{
    uint64_t acc = 0;
    if (valid) {
        if (in_smem) {
            const uint32_t *col = sU + lrow;
#pragma unroll 4
            for (int k = half; k < np; k += 2) mac<BIG>(acc, col[k * SSTRIDE], z[k], P.f);
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

// The true L values of one row (U~ read with a stride) into the pivot-order
// output LpC, using the per-column coefficients: 1x1: L_j = cA_j U_j; first
// column of a 2x2: L_j = cA_j U_{j+1} + cB_j U_j; second column:
// L_j = cA_j U_{j-1}.  Column j goes to position canon[j].
__device__ __forceinline__ void finish_row(const PanelParams &P, const uint32_t *u, int stride, int t, int np,
                                           const uint32_t *kind, const uint32_t *cA, const uint32_t *cB,
                                           const uint32_t *canon)
{
    uint32_t *g = P.LpC + t;
    for (int j = 0; j < np; ++j) {
        const uint32_t kd = kind[j];
        if (kd == K_1x1) {
            g[(int64_t)canon[j] * P.ldL] = fp_mul(cA[j], u[j * stride], P.f);
        } else if (kd == K_2A) {
            const uint32_t u0 = u[j * stride], u1 = u[(j + 1) * stride];
            g[(int64_t)canon[j] * P.ldL] = fp_add(fp_mul(cA[j], u1, P.f), fp_mul(cB[j], u0, P.f), P.f);
            g[(int64_t)canon[j + 1] * P.ldL] = fp_mul(cA[j + 1], u0, P.f);
            ++j;
        }
    }
}

// ---------------------------------------------------------------------------
// helper CTAs
// ---------------------------------------------------------------------------

// Post this CTA's answer to scan `sid`: the first row mn with a non-zero
// value (INT_MAX: none).  For a hit the row's U~ values (np of them) and the
// value x at it go to the scan's candidate slot first.  All compute threads.
__device__ __forceinline__ void post_answer(const PanelParams &P, Shared &sh, int lo, int sid, int mn, int np,
                                            uint32_t xval)
{
    const int tid = threadIdx.x;
    if (P.test_drop == 1) return;  // failure-detection test: the answer is never sent
    if (mn != INT_MAX) {
        const int lr = mn - lo;
        uint32_t *dst = P.partner_lp + ((int64_t)(sid % SCAN_RING) * MAX_PANEL_GRID + blockIdx.x) * PSTR;
        for (int k = tid; k < np; k += NCT)
            dst[k] = lr < SROWS ? sh.U[k * SSTRIDE + lr] : P.LpT[(int64_t)k * P.ldL + mn];
        if (tid == 0) dst[KP_MAX] = xval;
        __threadfence();
        cbar();
        if (tid == 0) {
            atomicMin(&P.scans[sid].min, mn);
            __threadfence();
            atomicOr(&P.scans[sid].mask[blockIdx.x >> 5], 1u << (blockIdx.x & 31));
            atomicAdd(&P.scans[sid].done, 1);
        }
    } else if (tid == 0) {
        atomicOr(&P.scans[sid].mask[blockIdx.x >> 5], 1u << (blockIdx.x & 31));
        atomicAdd(&P.scans[sid].done, 1);
    }
}

// CTA-wide minimum of v over the compute threads (all of them call it).
__device__ __forceinline__ int cta_min(Shared &sh, int v)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh.redi[warp] = v;
    cbar();
    int mn = INT_MAX;
    for (int i = 0; i < NCW; ++i) mn = min(mn, sh.redi[i]);
    cbar();
    return mn;
}

template <bool BIG>
__device__ void helper_cta(const PanelParams &P, Shared &sh, int lo, int hi)
{
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nrows = hi > lo ? hi - lo : 0;
    if (tid == 0) { sh.ev_ready = 0; sh.ev_done = 0; sh.quit = 0; sh.ev_fetched = 0; }
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
                if (kind == EV_END || kind == EV_FARPAIR) {
                    // these records carry up to 4*KP_MAX payload words
                    for (int k = 2 * KP_MAX / 4 + lane; k < EV_WORDS / 4; k += 32) ringv[k] = __ldcg(rec + 2 + k);
                    end = end || kind == EV_END;
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
                __syncwarp();
                if (gbuf_g[bi ^ 1] != g + 1) {
                    // prefetch the next group into the other buffer once nothing is in flight
                    if (last_g != g) asm volatile("cp.async.wait_group 0;" ::: "memory");
                    __syncwarp();
                    fetch_grp(g + 1, bi ^ 1);
                    last_g = g + 1;
                }
            }
            if (kind == EV_PIVOT2 || kind == EV_FARPAIR) {
                // S(t, b): for t > b one line per row, so all loads of the lane go
                // out before the first store (one round trip)
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
    for (int e = 0;; ++e) {
        if (tid == 0) {
            Spin sp;
            while (sh.ev_ready <= e && !sh.quit) {
                __nanosleep(32);
                if (sp.expired(2 * P.budget_ns + 1000000)) break;
            }
            sh.hgo = sh.ev_ready > e;  // one decision for every compute thread
        }
        cbar();
        if (!sh.hgo) return;  // quit or abort
        __threadfence_block();
        const int s = e % NSLOT;
        const int kind = sh.ev[s].kind;
        const int np = sh.ev[s].np, a = sh.ev[s].a, b = sh.ev[s].b, col = sh.ev[s].col;
        const uint32_t W = sh.ev[s].s0;
        const uint32_t *za = sh.ring[s];
        const uint32_t *zb = sh.ring[s] + KP_MAX;
        if (kind == EV_END) {
            // rewrite this CTA's rows as true L columns in pivot order
            const uint32_t *kinds = sh.ring[s];
            const uint32_t *cA = sh.ring[s] + KP_MAX;
            const uint32_t *cB = sh.ring[s] + 2 * KP_MAX;
            const uint32_t *canon = sh.ring[s] + 3 * KP_MAX;
            for (int lr = tid; lr < nrows; lr += NCT) {
                const int t = lo + lr;
                if (lr < SROWS) finish_row(P, sh.U + lr, SSTRIDE, t, np, kinds, cA, cB, canon);
                else finish_row(P, P.LpT + t, (int)P.ldL, t, np, kinds, cA, cB, canon);
            }
            return;
        }
        if (kind == EV_FARPAIR) {
            // the far pair's columns: c~_a from the scan's own column, c~_b by
            // a pass with z_b; then the rank-1 fixes of the later columns
            const int ncorr = sh.ev[s].aux & 0xffff, nres = sh.ev[s].aux >> 16;
            const uint32_t *corr = sh.ring[s] + KP_MAX;
            const uint32_t *resc = sh.ring[s] + EV_WORDS;
            const uint32_t *scP = P.scancol + (int64_t)(sh.ev[s].scan_id % SCAN_RING) * P.ldL;
            for (int base = 0; base < nrows; base += NCT / 2) {
                const int lr = base + (tid >> 1);
                const bool valid = lr < nrows;
                const bool sm = lr < SROWS;
                const int t = lo + lr;
                const uint32_t sb = valid ? (sm ? sh.scol[s][1][lr] : s_at(P.S, P.ldS, t, b)) : 0u;
                const uint32_t ubv = schur2<BIG>(P, sh.U, lr, t, sb, W, za, np, half, valid, sm);
                if (valid && half == 0) {
                    const uint32_t uav = scP[t];
                    if (sm) { sh.U[col * SSTRIDE + lr] = uav; sh.U[(col + 1) * SSTRIDE + lr] = ubv; }
                    P.LpT[(int64_t)col * P.ldL + t] = uav;
                    P.LpT[(int64_t)(col + 1) * P.ldL + t] = ubv;
                    for (int q = 0; q < ncorr; ++q) {
                        const int c = (int)corr[2 * q];
                        const uint32_t rho = corr[2 * q + 1];
                        uint32_t *gp = P.LpT + (int64_t)c * P.ldL + t;
                        const uint32_t old = sm ? sh.U[c * SSTRIDE + lr] : *gp;
                        const uint32_t nv = fp_sub(old, fp_mul(uav, rho, P.f), P.f);
                        if (sm) sh.U[c * SSTRIDE + lr] = nv;
                        *gp = nv;
                    }
                }
            }
            cbar();
            // the later scans, fixed and answered under their new ids
            for (int q = 0; q < nres; ++q) {
                const int so = (int)resc[-3 * (q + 1)], sn = (int)resc[-3 * (q + 1) + 1];
                const uint32_t rho = resc[-3 * (q + 1) + 2];
                const uint32_t *cold = P.scancol + (int64_t)(so % SCAN_RING) * P.ldL;
                uint32_t *cnew = P.scancol + (int64_t)(sn % SCAN_RING) * P.ldL;
                int firstnz = INT_MAX;
                for (int lr = tid; lr < nrows; lr += NCT) {
                    const int t = lo + lr;
                    const uint32_t uav = lr < SROWS ? sh.U[col * SSTRIDE + lr] : P.LpT[(int64_t)col * P.ldL + t];
                    const uint32_t c = fp_sub(cold[t], fp_mul(uav, rho, P.f), P.f);
                    cnew[t] = c;
                    if (c != 0 && t < firstnz) firstnz = t;
                }
                const int mn = cta_min(sh, firstnz);
                const uint32_t xv = mn != INT_MAX ? cnew[mn] : 0u;
                post_answer(P, sh, lo, sn, mn, col + 2, xv);
            }
            cbar();
            if (tid == 0) { __threadfence_block(); sh.ev_done = e + 1; }
            continue;
        }
        int firstnz = INT_MAX;
        uint32_t *cscan = (kind == EV_SCAN) ? P.scancol + (int64_t)(sh.ev[s].scan_id % SCAN_RING) * P.ldL : nullptr;
        for (int base = 0; base < nrows; base += NCT / 2) {
            const int lr = base + (tid >> 1);
            const bool valid = lr < nrows;
            const bool sm = lr < SROWS;
            const int t = lo + lr;
            const uint32_t sa = valid ? (sm ? sh.scol[s][0][lr] : s_at(P.S, P.ldS, t, a)) : 0u;
            if (kind == EV_PIVOT1) {
                const uint32_t c = schur2<BIG>(P, sh.U, lr, t, sa, W, za, np, half, valid, sm);
                if (valid && half == 0) {
                    if (sm) sh.U[col * SSTRIDE + lr] = c;
                    P.LpT[(int64_t)col * P.ldL + t] = c;
                }
            } else if (kind == EV_PIVOT2) {
                const uint32_t sb = valid ? (sm ? sh.scol[s][1][lr] : s_at(P.S, P.ldS, t, b)) : 0u;
                const uint32_t ca = schur2<BIG>(P, sh.U, lr, t, sa, W, za, np, half, valid, sm);
                const uint32_t cb = schur2<BIG>(P, sh.U, lr, t, sb, W, zb, np, half, valid, sm);
                if (valid && half == 0) {
                    if (sm) { sh.U[col * SSTRIDE + lr] = ca; sh.U[(col + 1) * SSTRIDE + lr] = cb; }
                    P.LpT[(int64_t)col * P.ldL + t] = ca;
                    P.LpT[(int64_t)(col + 1) * P.ldL + t] = cb;
                }
            } else {  // EV_SCAN: keep the column (a far pair reads it) and find its first non-zero
                const uint32_t c = schur2<BIG>(P, sh.U, lr, t, sa, W, za, np, half, valid, sm);
                if (valid && half == 0) cscan[t] = c;
                if (valid && c != 0 && t < firstnz) firstnz = t;
            }
        }
        if (kind == EV_SCAN) {
            const int mn = cta_min(sh, firstnz);
            const uint32_t xv = mn != INT_MAX ? cscan[mn] : 0u;
            post_answer(P, sh, lo, sh.ev[s].scan_id, mn, np, xv);
        }
        cbar();
        if (tid == 0) { __threadfence_block(); sh.ev_done = e + 1; }
    }
}

// ---------------------------------------------------------------------------
// leader CTA
// ---------------------------------------------------------------------------
template <bool BIG>
__device__ void leader_cta(const PanelParams &P, Shared &sh, bool helpers)
{
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const FieldP f = P.f;
    const int w = P.w;
    const int nh = gridDim.x - 1;
    for (int t = tid; t < W0; t += blockDim.x) sh.rinfo[t] = RI_UNDEC;
    for (int i = tid; i < SRING; i += blockDim.x) sh.res_ok[i] = 0;
    if (tid == 0) {
        sh.abort = 0; sh.ev_ready = 0; sh.ev_done = 0; sh.quit = 0;
        sh.nscan_pub = 0; sh.head_new = 0; sh.head_b = -1;
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
                if (kind == EV_END || kind == EV_FARPAIR) {
                    for (int k = lane; k < EV_WORDS; k += 32) rec[8 + k] = sh.ring[s][k];
                } else {
                    const int words = kind == EV_PIVOT2 ? 2 * KP_MAX : KP_MAX;
                    for (int k = lane; k < words; k += 32)
                        if (k % KP_MAX < np) rec[8 + k] = sh.ring[s][k];
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
                } else if (kind == EV_FARPAIR) {
                    const int nres = sh.ev[s].aux >> 16;
                    for (int q = 0; q < nres; ++q) {
                        const int sid = (int)sh.ring[s][EV_WORDS - 3 * (q + 1) + 1];
                        if (lane < 8) P.scans[sid].mask[lane] = 0u;
                        if (lane == 0) {
                            P.scans[sid].done = 0;
                            P.scans[sid].min = INT_MAX;
                        }
                        last_scan = sid > last_scan ? sid : last_scan;
                    }
                }
                end = end || (kind == EV_END);
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                atomicExch(&P.sync->ev_count, ready);
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
        const int chunk = (P.m - w + nh - 1) / nh;  // far rows per helper, as in helper_cta
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
    int ncol = 0, ia = 0, nscan = 0, ph = 0, pt = 0, ev_next = 0, nev = 0;
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
    // control warp (the last compute warp): settle the head of the FIFO.  Posts
    // head_new = the head after the answered scans that found no partner, and
    // head_b = the partner found by the scan there (-1: unanswered or none).
    auto resolved = [&](int id) { return ld_acquire_cta(&sh.res_ok[id % SRING]) == id + 1; };
    auto check_head = [&](bool wait) {
        __syncwarp();
        if (wait && ph < pt) {
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
        int v = -1;
        if (q < pt) {
            const int id = sh.pend_id[q % NPEND];
            if (resolved(id)) {  // the answer is read only after its flag
                res = true;
                v = sh.res_min[id % SRING];
                hit = v >= w && v < P.m;
            }
        }
        const unsigned miss = __ballot_sync(0xffffffffu, res && !hit);
        const int adv = __ffs(~miss) - 1;
        const int vb = __shfl_sync(0xffffffffu, hit ? v : -1, adv & 31);
        if (lane == 0) {
            sh.head_new = ph + adv;
            sh.head_b = vb;
        }
    };

    // A far scan found its partner: insert the far pair at the head of the
    // FIFO (all compute threads; ph is its index).
    auto handle_hit = [&](int b) {
        const int hs = ph % NPEND;
        const int aP = sh.pend_row[hs], sidP = sh.pend_id[hs], evP = sh.pend_ev[hs];
        const uint32_t Wsc = sh.pend_W[hs];
        const int chunk = (P.m - w + nh - 1) / nh;
        const int owner = 1 + (b - w) / chunk;
        const uint32_t *src = P.partner_lp + ((int64_t)(sidP % SCAN_RING) * MAX_PANEL_GRID + owner) * PSTR;
        uint32_t sbb = 0u;
        if (tid < ncol) sh.ub[tid] = __ldcg(src + tid);
        if (tid == 0) {
            sh.xy[0] = __ldcg(src + KP_MAX);
            sbb = s_at(P.S, P.ldS, b, b);
        }
        cbar();
        // z_b over the columns that precede row aP; far pairs weigh W / delta
        if (tid < ncol) {
            const int jb = tid - (sh.kind[tid] == K_2B);
            uint32_t zv = 0u;
            if (sh.brow[jb] < aP) {
                const uint32_t wt = sh.isfar[jb] ? fp_mul(Wsc, sh.invd[jb], f) : sh.pend_bw[hs][jb];
                zv = zval_w(tid, sh.ub, 1, sh, wt, f);
            }
            sh.zt[tid] = zv;
        }
        cbar();
        const uint32_t x = sh.xy[0];
        if (warp == 0) {
            // y~ = W S(b,b) - U~[b] . z_b
            uint64_t ay = 0;
            for (int k = lane; k < ncol; k += 32) mac<true>(ay, sh.ub[k], sh.zt[k], f);
            uint64_t sy = fp_reduce64(ay, f);
            for (int o = 16; o > 0; o >>= 1) sy += __shfl_xor_sync(0xffffffffu, sy, o);
            if (lane == 0) sh.xy[1] = fp_sub(fp_mul(Wsc, sbb, f), fp_reduce64(sy, f), f);
        }
        // the block's window column c~_b[t] for the window rows t >= aP (t < b)
        const bool rowb = inwin && lr >= aP;
        const uint32_t s_b = rowb ? __ldg(P.S + (int64_t)b * P.ldS + lr) : 0u;
        const uint32_t cb_t = schur2<BIG>(P, sh.U, lr, lr, s_b, Wsc, sh.zt, ncol, half, rowb, true);
        if (tid == 32) sh.xy[2] = fp_inv(fp_mul(Wsc, fp_mul(x, x, f), f), f);  // 1 / delta
        if (tid == NCT - 1) ring_ready(ev_next);
        cbar();
        const uint32_t y = sh.xy[1], invd = sh.xy[2];
        const int colP = ncol;
        if (rowb && half == 0) {
            sh.U[colP * SSTRIDE + lr] = 0u;  // c~_a = 0 on the window rows after aP
            sh.U[(colP + 1) * SSTRIDE + lr] = cb_t;
            P.LpT[(int64_t)colP * P.ldL + lr] = 0u;
            P.LpT[(int64_t)(colP + 1) * P.ldL + lr] = cb_t;
        }
        const int slot = ev_next % NSLOT;
        for (int k = tid; k < ncol; k += NCT) sh.ring[slot][k] = sh.zt[k];
        cbar();
        if (warp == 0) {
            // ---- the fixes of the later blocks' far columns (one warp) ----
            // rho_i = ext_i - sum_l rho_l z_i[c_l] over the corrected columns
            // c_l of earlier events; lanes hold the columns, each with the
            // block weight it had at the event being processed.
            int lcol[LPL], lkd[LPL];
            uint32_t lbw[LPL], lrho[LPL];
#pragma unroll
            for (int q = 0; q < LPL; ++q) { lcol[q] = 0; lkd[q] = 0; lbw[q] = 0u; lrho[q] = 0u; }
            int nl = 0, ncorr = 0, nres = 0;
            const uint32_t xe = fp_mul(x, invd, f);
            uint32_t *corr = sh.ring[slot] + KP_MAX;
            uint32_t *resc = sh.ring[slot] + EV_WORDS;
            auto rho_of = [&](int u, uint32_t We) -> uint32_t {
                // ext = z_u[colP] = x~ c~_b[u] W_e / delta  (c~_a[u] = 0)
                const uint32_t ext = fp_mul(fp_mul(xe, sh.U[(colP + 1) * SSTRIDE + u], f), We, f);
                uint64_t acc = 0;
#pragma unroll
                for (int q = 0; q < LPL; ++q) {
                    if (lane + 32 * q < nl) {
                        const int c = lcol[q];
                        uint32_t zc;
                        if (lkd[q] == K_1x1) zc = sh.U[c * SSTRIDE + u];
                        else if (lkd[q] == K_2A)
                            zc = fp_sub(fp_mul(sh.mx[c], sh.U[(c + 1) * SSTRIDE + u], f),
                                        fp_mul(sh.my[c], sh.U[c * SSTRIDE + u], f), f);
                        else zc = fp_mul(sh.mx[c - 1], sh.U[(c - 1) * SSTRIDE + u], f);
                        acc += fp_mul(lrho[q], fp_mul(zc, lbw[q], f), f);
                    }
                }
                uint64_t tot = fp_reduce64(acc, f);
                for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
                return fp_sub(ext, fp_reduce64(tot, f), f);
            };
            for (int e = evP + 1; e < nev; ++e) {
                const int es = e % EVT;
                const int ek = sh.evt_kind[es], u = sh.evt_u[es], ecol = sh.evt_col[es];
                const uint32_t We = sh.evt_W[es];
                if (ek == EK_SCAN) {
                    const uint32_t rho = rho_of(u, We);
                    const int so = sh.evt_sid[es], sn = nscan + nres;
                    __syncwarp();
                    if (lane == 0) {
                        resc[-3 * (nres + 1)] = (uint32_t)so;
                        resc[-3 * (nres + 1) + 1] = (uint32_t)sn;
                        resc[-3 * (nres + 1) + 2] = rho;
                        sh.evt_sid[es] = sn;
                        sh.pend_id[(ph + 1 + nres) % NPEND] = sn;
                    }
                    ++nres;
                    continue;
                }
                const uint32_t r0 = rho_of(u, We);
                const uint32_t r1 = (ek == EK_P2) ? rho_of(sh.evt_v[es], We) : 0u;
                if (lane == 0) {
                    corr[2 * ncorr] = (uint32_t)ecol;
                    corr[2 * ncorr + 1] = r0;
                    if (ek == EK_P2) {
                        corr[2 * ncorr + 2] = (uint32_t)(ecol + 1);
                        corr[2 * ncorr + 3] = r1;
                    }
                }
                ncorr += (ek == EK_P2) ? 2 : 1;
                // the event's block: older columns' weights grow by its delta,
                // its own columns start at the event's scale
                const uint32_t dl = sh.delta[ecol];
#pragma unroll
                for (int q = 0; q < LPL; ++q)
                    if (lane + 32 * q < nl) lbw[q] = fp_mul(lbw[q], dl, f);
                const int nadd = (ek == EK_P2) ? 2 : 1;
                for (int i = 0; i < nadd; ++i) {
                    const int l = nl + i;
                    if ((l & 31) == lane) {
#pragma unroll
                        for (int q = 0; q < LPL; ++q)
                            if (q == (l >> 5)) {
                                lcol[q] = ecol + i;
                                lkd[q] = (ek == EK_P1) ? K_1x1 : (i == 0 ? K_2A : K_2B);
                                lbw[q] = We;
                                lrho[q] = i == 0 ? r0 : r1;
                            }
                    }
                }
                nl += nadd;
            }
            if (lane == 0) { sh.ncorr = ncorr; sh.nres = nres; }
        }
        cbar();
        const int ncorr = sh.ncorr, nres = sh.nres;
        if (tid == 0) {
            sh.kind[colP] = K_2A; sh.kind[colP + 1] = K_2B;
            sh.isfar[colP] = 1; sh.isfar[colP + 1] = 1;
            sh.bw[colP] = fp_mul(W, invd, f);  // W / delta at the current scale
            sh.mx[colP] = x; sh.my[colP] = y; sh.piv[colP] = x; sh.w0[colP] = Wsc;
            sh.invd[colP] = invd; sh.delta[colP] = 0u;
            sh.brow[colP] = aP; sh.brow[colP + 1] = aP;
            sh.piv_rows[colP] = aP; sh.piv_rows[colP + 1] = b;
            sh.rinfo[aP] = RI_PIV + colP;
            P.consumed[b] = 1;
            Event &ev = sh.ev[slot];
            ev.kind = EV_FARPAIR; ev.a = aP; ev.b = b; ev.np = ncol; ev.s0 = Wsc; ev.col = colP;
            ev.scan_id = sidP; ev.aux = ncorr | (nres << 16);
            __threadfence_block();
            sh.ev_ready = ev_next + 1;
            sh.dbg[2] += 1;
            sh.dbg[3] += ncorr;
            sh.dbg[4] += nres;
        }
        ncol += 2;
        nscan += nres;
        ++ph;
        ++ev_next;
    };
    // settle the head: the answered misses become zero rows; a hit is inserted
    auto settle = [&](int hn, int hb) {
        for (int q = ph + tid; q < hn; q += NCT) sh.rinfo[sh.pend_row[q % NPEND]] = RI_ZERO;
        ph = hn;
        if (hb >= 0) handle_hit(hb);
        cbar();
    };

    for (;;) {
        const int np_pend = pt - ph;
        const bool room = ia < w && ncol + 2 * np_pend + 2 <= P.kp && ev_next < MAX_EVENTS - 64 &&
                          nscan < MAX_SCANS - 2 * NPEND - 2 &&
                          (np_pend == 0 || nev - sh.pend_ev[ph % NPEND] < EVT_LIM);
        if (!room) {
            if (ph == pt) break;  // nothing in flight: the panel is complete
            if (warp == NCW - 1) check_head(true);
            cbar();
            const int hn = sh.head_new, hb = sh.head_b;
            const bool ab = sh.abort;
            cbar();
            if (ab) break;
            settle(hn, hb);
            continue;
        }
        if (sh.rinfo[ia] != RI_UNDEC) {
            ++ia;
            continue;
        }
        const int a = ia;
        const int slot = ev_next % NSLOT;
        uint32_t *za = sh.ring[slot];
        uint32_t *zb = sh.ring[slot] + KP_MAX;
        if (tid < ncol) {
            ring_ready(ev_next);
            za[tid] = zval(tid, sh.U + a, SSTRIDE, sh, f);
        }
        if (warp == NCW - 1) {
            if (lane == 0) sh.dbg[0] += 1;
            check_head(false);
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
        cbar();
        {
            const int hn = sh.head_new, hb = sh.head_b;
            if (sh.abort) break;
            if (hb >= 0) {
                cbar();  // every thread has read the posted head
                settle(hn, hb);
                continue;  // the row is taken again
            }
            // misses only: mark their rows, nothing this row needs changes
            for (int q = ph + tid; q < hn; q += NCT) sh.rinfo[sh.pend_row[q % NPEND]] = RI_ZERO;
            ph = hn;
        }
        // Snapshot for this row's scan, should it issue one: a scan goes out
        // only while pt - ph < npend <= NPEND, so slot pt % NPEND then holds no
        // pending scan and always takes this row's weights.
        if (tid < ncol && pt - ph < NPEND) sh.pend_bw[pt % NPEND][tid] = sh.bw[tid];
        // c~_a[t] for the window rows t >= a (t = a included) and the first
        // non-zero of row a beyond a inside the window, in one pass
        const uint32_t ca_t = schur2<BIG>(P, sh.U, lr, lr, s_col, W, za, ncol, half, myrow, true);
        if (lr == a && half == 0) sh.caa = ca_t;
        int firstnz = (half == 0 && inwin && lr > a && ca_t != 0) ? lr : INT_MAX;
        for (int o = 16; o > 0; o >>= 1) firstnz = min(firstnz, __shfl_xor_sync(0xffffffffu, firstnz, o));
        if (lane == 0) sh.redi[warp] = firstnz;
        cbar();
        const uint32_t caa = sh.caa;

        if (caa != 0) {
            // ---- 1x1 pivot: U~[:, ncol] = c~_a, delta = W c~_a[a] ----
            if (myrow && half == 0) {
                sh.U[ncol * SSTRIDE + lr] = ca_t;
                P.LpT[(int64_t)ncol * P.ldL + lr] = ca_t;
            }
            const uint32_t delta = fp_mul(W, caa, f);
            if (tid < ncol && sh.kind[tid] != K_2B) sh.bw[tid] = fp_mul(sh.bw[tid], delta, f);
            if (tid == 0) {
                if (helpers) {
                    Event &ev = sh.ev[slot];
                    ev.kind = EV_PIVOT1; ev.a = a; ev.b = -1; ev.np = ncol; ev.s0 = W; ev.col = ncol;
                    ev.scan_id = 0; ev.aux = 0;
                    __threadfence_block();
                    sh.ev_ready = ev_next + 1;
                }
                sh.kind[ncol] = K_1x1; sh.isfar[ncol] = 0; sh.bw[ncol] = W; sh.piv[ncol] = caa; sh.w0[ncol] = W;
                sh.delta[ncol] = delta; sh.brow[ncol] = a;
                sh.piv_rows[ncol] = a;
                sh.rinfo[a] = RI_PIV + ncol;
                const int es = nev % EVT;
                sh.evt_kind[es] = EK_P1; sh.evt_u[es] = a; sh.evt_v[es] = -1; sh.evt_col[es] = ncol;
                sh.evt_sid[es] = -1; sh.evt_W[es] = W;
            }
            W = fp_mul(W, delta, f);
            ++ncol;
            ++ia;
            ++nev;
            if (helpers) ++ev_next;
            cbar();
            continue;
        }

        int b = INT_MAX;
        for (int i = 0; i < NCW; ++i) b = min(b, sh.redi[i]);
        if (b == INT_MAX && helpers) {
            // ---- far scan: publish it and go on as if the row were zero ----
            if (pt - ph >= P.npend) {
                if (warp == NCW - 1) check_head(true);
                cbar();
                const int hn = sh.head_new, hb = sh.head_b;
                const bool ab = sh.abort;
                cbar();
                if (ab) break;
                settle(hn, hb);
                continue;  // the row is taken again from the top
            }
            if (tid == NCT - 1) {
                Event &ev = sh.ev[slot];
                ev.kind = EV_SCAN; ev.a = a; ev.b = -1; ev.np = ncol; ev.s0 = W; ev.col = -1;
                ev.scan_id = nscan; ev.aux = 0;
                const int ps = pt % NPEND;
                sh.pend_id[ps] = nscan; sh.pend_row[ps] = a; sh.pend_ev[ps] = nev; sh.pend_W[ps] = W;
                sh.rinfo[a] = RI_PEND;
                const int es = nev % EVT;
                sh.evt_kind[es] = EK_SCAN; sh.evt_u[es] = a; sh.evt_v[es] = -1; sh.evt_col[es] = -1;
                sh.evt_sid[es] = nscan; sh.evt_W[es] = W;
                sh.dbg[5] += 1;
                __threadfence_block();
                sh.ev_ready = ev_next + 1;
            }
            ++nscan;
            ++pt;
            ++ia;
            ++ev_next;
            ++nev;
            cbar();
            continue;
        }
        if (b == INT_MAX) {
            // ---- zero row (no far rows to search) ----
            if (tid == 0) sh.rinfo[a] = RI_ZERO;
            ++ia;
            cbar();
            continue;
        }

        // ---- 2x2 pivot on (a, b), both in the window ----
        uint32_t s_ab = 0u, s_bb = 0u;
        if (tid == 0) {
            s_ab = s_at(P.S, P.ldS, a, b);
            s_bb = s_at(P.S, P.ldS, b, b);
        }
        if (tid < ncol) sh.ub[tid] = sh.U[tid * SSTRIDE + b];
        cbar();
        if (tid < ncol) zb[tid] = zval(tid, sh.ub, 1, sh, f);
        cbar();
        // x~ = W S(a,b) - U~[b] . z_a ;  y~ = W S(b,b) - U~[b] . z_b   (warp 0)
        if (warp == 0) {
            uint64_t ax = 0, ay = 0;
            for (int k = lane; k < ncol; k += 32) {
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
        const uint32_t cb_t = schur2<BIG>(P, sh.U, lr, lr, s_b, W, zb, ncol, half, myrow, true);
        cbar();
        const uint32_t x = sh.xy[0], y = sh.xy[1];
        if (myrow && half == 0) {
            sh.U[ncol * SSTRIDE + lr] = ca_t;  // c~_a[a] = 0 here
            sh.U[(ncol + 1) * SSTRIDE + lr] = cb_t;
            P.LpT[(int64_t)ncol * P.ldL + lr] = ca_t;
            P.LpT[(int64_t)(ncol + 1) * P.ldL + lr] = cb_t;
        }
        const uint32_t delta = fp_mul(W, fp_mul(x, x, f), f);
        if (tid < ncol && sh.kind[tid] != K_2B) sh.bw[tid] = fp_mul(sh.bw[tid], delta, f);
        if (tid == 0) {
            if (helpers) {
                Event &ev = sh.ev[slot];
                ev.kind = EV_PIVOT2; ev.a = a; ev.b = b; ev.np = ncol; ev.s0 = W; ev.col = ncol;
                ev.scan_id = 0; ev.aux = 0;
                __threadfence_block();
                sh.ev_ready = ev_next + 1;
            }
            sh.kind[ncol] = K_2A; sh.kind[ncol + 1] = K_2B; sh.isfar[ncol] = 0; sh.isfar[ncol + 1] = 0;
            sh.bw[ncol] = W; sh.mx[ncol] = x; sh.my[ncol] = y; sh.piv[ncol] = x; sh.w0[ncol] = W;
            sh.delta[ncol] = delta; sh.brow[ncol] = a; sh.brow[ncol + 1] = a;
            sh.piv_rows[ncol] = a; sh.piv_rows[ncol + 1] = b;
            sh.rinfo[a] = RI_PIV + ncol;
            sh.rinfo[b] = RI_PART;
            P.consumed[b] = 1;
            const int es = nev % EVT;
            sh.evt_kind[es] = EK_P2; sh.evt_u[es] = a; sh.evt_v[es] = b; sh.evt_col[es] = ncol;
            sh.evt_sid[es] = -1; sh.evt_W[es] = W;
        }
        W = fp_mul(W, delta, f);
        ncol += 2;
        ++ia;
        ++nev;
        if (helpers) ++ev_next;
        cbar();
    }
    const int iend = ia;
    cbar();

    // ---- end of panel: batch inversion, true D and the L coefficients ----
    const bool aborted = sh.abort != 0;
    if (!aborted) {
        if (tid == 0) {
            // per block: its pivot value and its scale, inverted together (Montgomery's trick)
            int nv = 0;
            for (int j = 0; j < ncol; ++j)
                if (sh.kind[j] != K_2B) { sh.bi[nv++] = sh.piv[j]; sh.bi[nv++] = sh.w0[j]; }
            uint32_t run = 1;
            for (int i = 0; i < nv; ++i) { run = fp_mul(run, sh.bi[i], f); sh.bpre[i] = run; }
            uint32_t inv = nv ? fp_inv(run, f) : 1u;
            for (int i = nv - 1; i >= 0; --i) {
                const uint32_t before = i ? sh.bpre[i - 1] : 1u;
                const uint32_t vi = sh.bi[i];
                sh.bi[i] = fp_mul(inv, before, f);  // inverse of value i
                inv = fp_mul(inv, vi, f);
            }
            int v = 0;
            for (int j = 0; j < ncol; ++j) {
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
        // pivot order: the blocks by their first window row, the zero rows
        // ascending (block-wide prefix sums over the window rows)
        {
            const int t = tid;  // one thread per window row (NCT >= W0)
            const int ri = (t < iend && t < W0) ? sh.rinfo[t] : RI_UNDEC;
            const int cnt = ri >= RI_PIV ? (sh.kind[ri - RI_PIV] == K_1x1 ? 1 : 2) : 0;
            const int zf = ri == RI_ZERO ? 1 : 0;
            int ic = cnt, iz = zf;
            for (int o = 1; o < 32; o <<= 1) {
                const int vc = __shfl_up_sync(0xffffffffu, ic, o), vz = __shfl_up_sync(0xffffffffu, iz, o);
                if (lane >= o) { ic += vc; iz += vz; }
            }
            if (lane == 31) { sh.redi[warp] = ic; sh.redj[warp] = iz; }
            cbar();
            int oc = 0, oz = 0;
            for (int i = 0; i < warp; ++i) { oc += sh.redi[i]; oz += sh.redj[i]; }
            const int pos = oc + ic - cnt, zpos = oz + iz - zf;
            if (cnt) {
                const int col = ri - RI_PIV;
                sh.canon[col] = pos;
                if (cnt == 2) sh.canon[col + 1] = pos + 1;
            }
            if (zf) {
                P.out->zero_rows[zpos] = t;
                P.out->zero_np[zpos] = pos;
            }
            if (tid == NCT - 1) sh.xy[3] = (uint32_t)(oz + iz);  // zero rows
        }
        cbar();
        for (int j = tid; j < ncol; j += NCT) {
            const int k = sh.canon[j];
            P.out->piv_rows[k] = sh.piv_rows[j];
            P.out->dval[k] = sh.dtrue[j];
            P.out->eval[k] = sh.etrue[j];
        }
        if (helpers) {
            // the end event carries the column kinds, the true-L coefficients and the order
            const int slot = ev_next % NSLOT;
            if (tid < ncol) {
                ring_ready(ev_next);
                sh.ring[slot][tid] = sh.kind[tid];
                sh.ring[slot][KP_MAX + tid] = sh.cA[tid];
                sh.ring[slot][2 * KP_MAX + tid] = sh.cB[tid];
                sh.ring[slot][3 * KP_MAX + tid] = (uint32_t)sh.canon[tid];
            }
            if (tid == 0) ring_ready(ev_next);
            cbar();
            if (tid == 0) {
                Event &ev = sh.ev[slot];
                ev.kind = EV_END; ev.a = -1; ev.b = -1; ev.np = ncol; ev.s0 = 0; ev.col = -1;
                ev.scan_id = 0; ev.aux = 0;
                __threadfence_block();
                sh.ev_ready = ev_next + 1;
            }
        }
        // rewrite the window rows as true L columns in pivot order
        for (int k = tid; k < ncol; k += NCT) {
            sh.bi[k] = sh.kind[k];
            sh.bpre[k] = (uint32_t)sh.canon[k];
        }
        cbar();
        for (int t = tid; t < w; t += NCT)
            finish_row(P, sh.U + t, SSTRIDE, t, ncol, sh.bi, sh.cA, sh.cB, sh.bpre);
    }
    cbar();
    if (tid == 0) { __threadfence_block(); sh.quit = 1; }
    __threadfence();
    cbar();

    // ---- compaction of the remaining rows [iend, m) minus consumed partners ----
    const int m = P.m;
    const int len = m - iend;
    const int per = (len + NCT - 1) / NCT;
    const int clo = iend + tid * per, chi = min(m, clo + per);
    int cnt = 0;
    for (int t = clo; t < chi; ++t) cnt += P.consumed[t] ? 0 : 1;
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
    for (int t = clo; t < chi; ++t) {
        if (!P.consumed[t]) {
            P.sigma[pos] = t;
            P.idx_next[pos] = P.idx[t];
            ++pos;
        }
    }
    if (tid == 0) {
        P.out->np = aborted ? 0 : ncol;
        P.out->nzero = aborted ? 0 : (int)sh.xy[3];
        P.out->iend = iend;
        P.out->m_next = total;
        P.out->abort = (aborted ? 1 : 0) | *((volatile int *)&P.sync->abort);
        P.out->nscan = nscan;
        for (int i = 0; i < 8; ++i) P.out->cyc[i] = 0;
        for (int i = 0; i < 16; ++i) P.out->dbg[i] = sh.dbg[i];
    }
}

template <bool BIG>
__global__ void __launch_bounds__(BLOCK, 1) panel_kernel(PanelParams P)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    Shared &sh = *reinterpret_cast<Shared *>(smem_raw);
    const bool helpers = gridDim.x > 1;
    if (*(volatile int32_t *)P.status != 0) {
        // an earlier kernel of this factorisation gave up: end it here
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            P.out->np = 0; P.out->nzero = 0; P.out->iend = 0; P.out->m_next = 0;
            P.out->abort = 1; P.out->nscan = 0;
        }
        return;
    }
    if (blockIdx.x == 0) {
        leader_cta<BIG>(P, sh, helpers);
    } else {
        const int nh = gridDim.x - 1;
        const int far = P.m - P.w;
        const int chunk = (far + nh - 1) / nh;
        const int lo = P.w + (blockIdx.x - 1) * chunk;
        const int hi = min(P.m, lo + chunk);
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
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(BLOCK), args, smem, st);
}
