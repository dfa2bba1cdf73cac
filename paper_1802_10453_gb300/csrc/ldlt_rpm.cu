// ldlt_rpm.cu -- host side of the C ABI declared in include/ldlt_rpm.h.
//
// Blocked right-looking form of the lexicographic elimination (Algorithm 4's
// pivot order, Algorithm 2's level-3 updates):
//   ingest:   S = lower(A) mod p, compact index = original index
//   repeat:   panel   -- pivot chain over the first W0 rows of S (panel.cu):
//                        up to KP_MAX pivots, their L columns for every row;
//                        pivots, D and zero rows appended to the global lists
//             store   -- L columns into Lw (by original row)
//             update  -- S <- S[sigma, sigma] - G D G^T on the remaining rows
//                        (SYRDK, FP64 or tensor-core form), rows compacted
//   finalize: A <- L in perm order with D on the diagonal (PERM)
// The loop runs on the device: every kernel of a panel step reads its sizes
// from the loop state and the panel record in device memory, and the steps
// are one CUDA graph whose while node repeats them until the loop state says
// the factorisation has ended.  A call enqueues that graph (built on the
// first call with the same arguments, then reused) and returns; nothing is
// read back.  With profiling on, the same kernels are launched from a host
// loop that reads the record after each panel to time the phases.
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/ldlt_rpm.h"
#include "ldlt_internal.cuh"

namespace {

int64_t g_budget_ns = 2000000000LL;
int g_npend = LDLT_SPECULATION_DEFAULT;  // far scans in flight
int g_test_drop = 0;  // failure-detection tests: LDLT_TEST_DROP_*

// ---- profiling (optional) --------------------------------------------------
struct Prof {
    bool on = false;
    double acc[32] = {};
    double hbm[16] = {};     // see ldlt_rpm_profile_read_hbm
    // panel start, after the panel, after the L scatter, after the operand
    // split, after the update; ingest and finalize start / end
    cudaEvent_t ev[5] = {};
    cudaEvent_t evh[4] = {};
    bool ready = false;
};
Prof g_prof;

void prof_init()
{
    if (!g_prof.ready) {
        for (auto &e : g_prof.ev) cudaEventCreate(&e);
        for (auto &e : g_prof.evh) cudaEventCreate(&e);
        g_prof.ready = true;
    }
}

// Accumulate the phase times of the panel step just completed (the caller
// synchronised the stream after its last event).
void prof_collect()
{
    cudaEvent_t *ev = g_prof.ev;
    float t[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]);
    g_prof.acc[0] += t[0];
    g_prof.acc[1] += t[1] + t[2];
    g_prof.acc[2] += t[3];
    g_prof.hbm[2] += t[1];
    g_prof.hbm[3] += t[2];
}

uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }

uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod64(r, a, m);
        a = mulmod64(a, a, m);
        e >>= 1;
    }
    return r;
}

// Deterministic Miller-Rabin: bases 2, 3, 5, 7 decide every n < 3,215,031,751.
bool is_prime_u32(uint32_t n)
{
    if (n < 2) return false;
    for (uint32_t q : {2u, 3u, 5u, 7u}) {
        if (n == q) return true;
        if (n % q == 0) return false;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint64_t a : {2ull, 3ull, 5ull, 7ull}) {
        uint64_t x = powmod64(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mulmod64(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

int fp64_kred(uint32_t p)
{
    const double h = (double)((p - 1) / 2);
    const double lim = 9007199254740992.0 - 1.5 * (double)p;
    const double q = h * h > 1.0 ? h * h : 1.0;
    double k = lim / q;
    return k >= 1.0 ? (k > 1e9 ? 1000000000 : (int)k) : 0;
}

struct Layout {
    int64_t ldS;
    size_t S0, S1, Lw, LpT, LpC, idx0, idx1, sigma, consumed, piv_all, d_all, e_all, zero_all, zero_cols;
    size_t out, sync, loop, evlog, scans, partner_lp, scancol, zlog, opA, opB, total;
};


int make_layout(int64_t n, uint32_t p, int path, Layout &L)
{
    const int64_t nn = n > 0 ? n : 1;
    L.ldS = round_up(nn, 64);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (size_t)round_up((int64_t)bytes, 256);
        return o;
    };
    const size_t mat = (size_t)nn * (size_t)L.ldS * 4;
    L.S0 = take(mat);
    L.S1 = take(mat);
    L.Lw = take(mat);
    L.LpT = take((size_t)KP_MAX * (size_t)L.ldS * 4);
    L.LpC = take((size_t)KP_MAX * (size_t)L.ldS * 4);
    L.idx0 = take((size_t)nn * 4);
    L.idx1 = take((size_t)nn * 4);
    L.sigma = take((size_t)nn * 4);
    L.consumed = take((size_t)nn);
    L.piv_all = take((size_t)nn * 4);
    L.d_all = take((size_t)nn * 4);
    L.e_all = take((size_t)nn * 4);
    L.zero_all = take((size_t)nn * 4);
    L.zero_cols = take((size_t)nn * 4);
    L.out = take(sizeof(PanelOut));
    L.sync = take(sizeof(PanelSync));
    L.loop = take(sizeof(LoopState));
    L.evlog = take((size_t)MAX_EVENTS * EV_REC * 4);
    L.scans = take((size_t)MAX_SCANS * sizeof(ScanSlot));
    L.partner_lp = take((size_t)SCAN_RING * MAX_PANEL_GRID * PSTR * 4);
    L.scancol = take((size_t)SCAN_RING * (size_t)L.ldS * 4);
    L.zlog = take((size_t)ZLOG_EV * 2 * KP_MAX * 4);
    if (path == LDLT_PATH_FP64) {
        L.opA = take(fp64_operand_bytes(nn));
        L.opB = L.opA;  // GT follows GDT inside the same allocation
    } else {
        const int limbs = tc_limbs(p);
        L.opA = take(tc_operand_bytes(nn, limbs));
        L.opB = L.opA;
    }
    L.total = off;
    return LDLT_OK;
}

int check_args(int64_t n, uint32_t p, int path)
{
    if (n < 0 || n > (int64_t)1 << 30) return LDLT_ERR_ARG;
    if (path != LDLT_PATH_FP64 && path != LDLT_PATH_TC) return LDLT_ERR_ARG;
    if (p >= (1u << 31)) return LDLT_ERR_P_RANGE;
    if (!is_prime_u32(p)) return LDLT_ERR_NOT_PRIME;
    if (path == LDLT_PATH_FP64 && fp64_kred(p) < 1) return LDLT_ERR_P_RANGE;
    if (path == LDLT_PATH_TC && tc_limbs(p) < 1) return LDLT_ERR_P_RANGE;
    return LDLT_OK;
}

#define CK(call)                                \
    do {                                        \
        cudaError_t _e = (call);                \
        if (_e != cudaSuccess) return LDLT_ERR_CUDA; \
    } while (0)

}  // namespace

extern "C" int ldlt_rpm_version(void) { return 10000; }

extern "C" void ldlt_rpm_profile_enable(int on)
{
    g_prof.on = on != 0;
    if (g_prof.on) prof_init();
}

extern "C" void ldlt_rpm_profile_reset(void)
{
    for (double &a : g_prof.acc) a = 0.0;
    for (double &a : g_prof.hbm) a = 0.0;
}

extern "C" int ldlt_rpm_profile_read(double out[32])
{
    if (!out) return LDLT_ERR_ARG;
    for (int i = 0; i < 32; ++i) out[i] = g_prof.acc[i];
    return LDLT_OK;
}

extern "C" int ldlt_rpm_profile_read_hbm(double out[16])
{
    if (!out) return LDLT_ERR_ARG;
    for (int i = 0; i < 16; ++i) out[i] = g_prof.hbm[i];
    return LDLT_OK;
}

extern "C" void ldlt_rpm_set_wait_budget_ns(int64_t ns) { g_budget_ns = ns > 0 ? ns : 2000000000LL; }

extern "C" int ldlt_rpm_set_speculation(int depth)
{
    if (depth < 1 || depth > 16) return LDLT_ERR_ARG;
    g_npend = depth;
    return LDLT_OK;
}

extern "C" int ldlt_rpm_test_drop(int which)
{
    if (which != 0 && which != LDLT_TEST_DROP_SCAN_ANSWERS && which != LDLT_TEST_DROP_UPDATE_COPIES)
        return LDLT_ERR_ARG;
    g_test_drop = which;
    return LDLT_OK;
}

extern "C" int ldlt_rpm_workspace_bytes(int64_t n, uint32_t p, int path, size_t *bytes)
{
    if (!bytes) return LDLT_ERR_ARG;
    int rc = check_args(n, p, path);
    if (rc != LDLT_OK) return rc;
    Layout L;
    make_layout(n, p, path, L);
    *bytes = L.total;
    return LDLT_OK;
}

extern "C" int ldlt_rpm_factor(int64_t n, uint32_t p, uint32_t *A, int64_t lda, int32_t *perm,
                               uint32_t *e, int64_t *rank, int32_t *status, int path, void *ws,
                               size_t ws_bytes, void *stream)
{
    return factor_core(n, p, A, lda, perm, e, rank, status, path, ws, ws_bytes, stream, nullptr, nullptr);
}

namespace {

// Everything the kernels of one factorisation are launched with.  The two
// halves of a loop iteration run panels from S0 into S1 and back, so each
// launch's arguments are fixed and the loop can be a graph.
struct Plan {
    int64_t n, lda, ldS;
    uint32_t p;
    int path, nsm, limbs, pgrid;
    uint32_t *A;
    int32_t *perm, *status;
    uint32_t *e;
    int64_t *rank;
    const int32_t *gperm;
    int *gbad;
    FieldP f;
    uint32_t *Sbuf[2], *Lw, *LpT, *LpC;
    int *idxb[2], *sigma, *piv_all, *zero_all, *zero_cols;
    uint32_t *d_all, *e_all;
    uint8_t *consumed, *opA, *opB;
    PanelOut *out;
    PanelSync *sync;
    LoopState *ls;
    PanelParams pp[2];
};

void plan_make(Plan &c, int64_t n, uint32_t p, int path, uint32_t *A, int64_t lda, int32_t *perm, uint32_t *e,
               int64_t *rank, int32_t *status, void *ws, const int32_t *gperm, int *gbad, const Layout &Lo, int nsm)
{
    uint8_t *w = (uint8_t *)ws;
    c.n = n; c.lda = lda; c.ldS = Lo.ldS; c.p = p; c.path = path; c.nsm = nsm;
    c.limbs = (path == LDLT_PATH_TC) ? tc_limbs(p) : 0;
    c.A = A; c.perm = perm; c.status = status; c.e = e; c.rank = rank; c.gperm = gperm; c.gbad = gbad;
    c.f = make_field(p);
    c.Sbuf[0] = (uint32_t *)(w + Lo.S0);
    c.Sbuf[1] = (uint32_t *)(w + Lo.S1);
    c.Lw = (uint32_t *)(w + Lo.Lw);
    c.LpT = (uint32_t *)(w + Lo.LpT);
    c.LpC = (uint32_t *)(w + Lo.LpC);
    c.idxb[0] = (int *)(w + Lo.idx0);
    c.idxb[1] = (int *)(w + Lo.idx1);
    c.sigma = (int *)(w + Lo.sigma);
    c.consumed = w + Lo.consumed;
    c.piv_all = (int *)(w + Lo.piv_all);
    c.d_all = (uint32_t *)(w + Lo.d_all);
    c.e_all = (uint32_t *)(w + Lo.e_all);
    c.zero_all = (int *)(w + Lo.zero_all);
    c.zero_cols = (int *)(w + Lo.zero_cols);
    c.out = (PanelOut *)(w + Lo.out);
    c.sync = (PanelSync *)(w + Lo.sync);
    c.ls = (LoopState *)(w + Lo.loop);
    c.opA = w + Lo.opA;
    c.opB = c.opA;
    if (path == LDLT_PATH_TC)
        c.opB = c.opA + (size_t)round_up(round_up(n, 128) * (int64_t)c.limbs * KP_MAX * 2, 256);
    // the first panel is the largest: its grid serves every later panel
    c.pgrid = panel_grid((int)n, nsm < MAX_PANEL_GRID ? nsm : MAX_PANEL_GRID);
    for (int h = 0; h < 2; ++h) {
        PanelParams &pp = c.pp[h];
        pp.S = c.Sbuf[h]; pp.ldS = c.ldS; pp.ls = c.ls; pp.f = c.f; pp.kp = KP_MAX;
        pp.LpT = c.LpT; pp.LpC = c.LpC; pp.ldL = c.ldS;
        pp.consumed = c.consumed; pp.idx = c.idxb[h]; pp.sigma = c.sigma; pp.idx_next = c.idxb[h ^ 1];
        pp.out = c.out; pp.sync = c.sync;
        pp.piv_all = c.piv_all; pp.d_all = c.d_all; pp.e_all = c.e_all;
        pp.zero_all = c.zero_all; pp.zero_cols = c.zero_cols;
        pp.evlog = (uint32_t *)(w + Lo.evlog);
        pp.scans = (ScanSlot *)(w + Lo.scans);
        pp.partner_lp = (uint32_t *)(w + Lo.partner_lp);
        pp.scancol = (uint32_t *)(w + Lo.scancol);
        pp.zlog = (uint32_t *)(w + Lo.zlog);
        pp.budget_ns = g_budget_ns; pp.status = status;
        pp.npend = g_npend;
        pp.test_drop = g_test_drop;
    }
}

// status = 0, S = lower(A) mod p (or P^T A P), loop state at order n.
// ev (profiling) brackets the ingest.
cudaError_t enqueue_start(const Plan &c, cudaStream_t st, cudaEvent_t *ev = nullptr)
{
    cudaError_t err = cudaMemsetAsync(c.status, 0, sizeof(int32_t), st);
    if (err != cudaSuccess) return err;
    if (ev && (err = cudaEventRecord(ev[0], st)) != cudaSuccess) return err;
    err = c.gperm ? launch_ingest_perm(c.A, c.lda, c.n, c.gperm, c.Sbuf[0], c.ldS, c.idxb[0], c.f, c.gbad, st)
                  : launch_ingest(c.A, c.lda, c.n, c.Sbuf[0], c.ldS, c.idxb[0], c.f, st);
    if (err != cudaSuccess) return err;
    if (ev && (err = cudaEventRecord(ev[1], st)) != cudaSuccess) return err;
    return launch_loop_step(c.ls, c.out, 1, c.n, c.status, c.consumed, c.sync, 0, 0, c.nsm, st);
}

// One panel step on half h: pivot chain (which also appends to the pivot and
// zero-row lists), L columns, operand split, level-3 update (the split does
// the compaction of a panel without pivots), loop advance.  ev (profiling):
// panel start, panel end, scatter end, split end, update end.
cudaError_t enqueue_step(const Plan &c, int h, cudaGraphConditionalHandle cond, int set_cond, cudaEvent_t *ev,
                         cudaStream_t st)
{
#define EQ(call)                                 \
    do {                                         \
        cudaError_t _e = (call);                 \
        if (_e != cudaSuccess) return _e;        \
    } while (0)
    if (ev) EQ(cudaEventRecord(ev[0], st));
    EQ(launch_panel(c.pp[h], c.pgrid, st));
    if (ev) EQ(cudaEventRecord(ev[1], st));
    EQ(launch_lw_scatter(c.LpC, c.ldS, c.n, c.ls, c.out, c.idxb[h], c.Lw, c.ldS, st));
    if (ev) EQ(cudaEventRecord(ev[2], st));
    if (c.path == LDLT_PATH_FP64) {
        double *GDT = (double *)c.opA;
        double *GT = GDT + (size_t)KP_MAX * c.ldS;
        EQ(launch_split_fp64(c.LpC, c.ldS, c.sigma, c.n, c.ls, c.out, c.f, GDT, GT, c.ldS, c.Sbuf[h], c.ldS,
                             c.Sbuf[h ^ 1], st));
        if (ev) EQ(cudaEventRecord(ev[3], st));
        EQ(launch_syrdk_fp64(c.Sbuf[h], c.ldS, c.sigma, c.n, c.ls, c.out, GDT, GT, c.ldS, c.f, c.Sbuf[h ^ 1], st));
    } else {
        EQ(launch_split_tc(c.LpC, c.ldS, c.sigma, c.n, c.ls, c.out, c.f, c.limbs, c.opA, c.opB, c.Sbuf[h], c.ldS,
                           c.Sbuf[h ^ 1], st));
        if (ev) EQ(cudaEventRecord(ev[3], st));
        EQ(launch_syrdk_tc(c.Sbuf[h], c.ldS, c.sigma, c.ls, c.out, c.opA, c.opB, c.limbs, c.f, c.Sbuf[h ^ 1],
                           g_budget_ns, c.status, c.nsm, g_test_drop == LDLT_TEST_DROP_UPDATE_COPIES, st));
    }
    if (ev) EQ(cudaEventRecord(ev[4], st));
    EQ(launch_loop_step(c.ls, c.out, 0, c.n, c.status, c.consumed, c.sync, cond, set_cond, c.nsm, st));
    return cudaSuccess;
#undef EQ
}

cudaError_t enqueue_finish(const Plan &c, cudaStream_t st, cudaEvent_t *ev = nullptr)
{
    cudaError_t err;
    if (ev && (err = cudaEventRecord(ev[0], st)) != cudaSuccess) return err;
    err = launch_finalize(c.n, c.Lw, c.ldS, c.piv_all, c.d_all, c.e_all, c.zero_all, c.zero_cols, c.ls, c.A,
                          c.lda, c.perm, c.e, c.rank, st);
    if (err != cudaSuccess) return err;
    if (ev && (err = cudaEventRecord(ev[1], st)) != cudaSuccess) return err;
    return cudaSuccess;
}

// Profiling: the same kernels from a host loop, one readback per panel.
int run_profiled(const Plan &c, cudaStream_t st)
{
    double *hb = g_prof.hbm;
    const double tri = (double)c.n * (double)(c.n + 1) * 0.5;
    CK(enqueue_start(c, st, g_prof.evh));
    g_prof.acc[5] += 2;  // ingest, loop start
    hb[4] += 1;
    hb[8] += 8.0 * tri;  // lower triangle of A read, of S written
    int m = (int)c.n;
    int nupd = 0;  // update launches of this call
    int lb = 0, la = 0, ash = 8;
    if (c.path == LDLT_PATH_TC) { lb = c.limbs; la = tc_limbs_a(c.p, &ash); }
    for (int ipanel = 0;; ++ipanel) {
        CK(enqueue_step(c, ipanel & 1, 0, 0, g_prof.ev, st));
        struct { int h[8]; long long cyc[8]; long long dbg[16]; } rb;
        static_assert(offsetof(PanelOut, cyc) == 8 * sizeof(int), "PanelOut layout");
        LoopState lh;
        CK(cudaMemcpyAsync(&rb, c.out, sizeof(rb), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&lh, c.ls, sizeof(lh), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        prof_collect();
        const int *hdr = rb.h;
        const int np = hdr[0], m_next = hdr[3];
        g_prof.acc[5] += 5;  // panel, L scatter, split, update, loop step
        g_prof.acc[6] += 1;
        g_prof.acc[7] += hdr[5];
        for (int i = 0; i < 8; ++i) g_prof.acc[8 + i] += (double)rb.cyc[i];
        for (int i = 0; i < 16; ++i) g_prof.acc[16 + i] += (double)rb.dbg[i];
        if (!hdr[4] && np > 0 && m_next > 0) {
            g_prof.acc[3] += (double)m_next * (double)(m_next + 1) * 0.5 * (double)np;
            g_prof.acc[4] += 1;
        }
        if (!hdr[4] && np > 0) {
            hb[6] += 1;
            hb[10] += 8.0 * (double)np * (double)m;  // np L columns of m rows read, written by row
            if (m_next > 0) {
                const double kpad = (double)round_up(np, 64), rows = (double)round_up(m_next, 128);
                hb[7] += 1;
                hb[11] += 4.0 * (double)np * (double)m_next;  // the columns of the remaining rows
                const double ops = c.path == LDLT_PATH_TC ? 2.0 * rows * la * kpad * (1.0 + lb)  // A' and B'
                                                          : 2.0 * 8.0 * kpad * (double)c.ldS;     // GD^T and G^T
                hb[11] += ops;
                // the update: the old lower triangle read and the new one written, the operands read once
                hb[12] += 8.0 * (double)m_next * (double)(m_next + 1) * 0.5 + ops;
                hb[13] += 1;
                if (nupd++ < 3) hb[14] += 8.0 * (double)m_next * (double)(m_next + 1) * 0.5 + ops;
            }
        }
        m = m_next;
        if (lh.done) break;
    }
    CK(enqueue_finish(c, st, g_prof.evh + 2));
    g_prof.acc[5] += 1;
    CK(cudaStreamSynchronize(st));
    float ti = 0, tf = 0;
    cudaEventElapsedTime(&ti, g_prof.evh[0], g_prof.evh[1]);
    cudaEventElapsedTime(&tf, g_prof.evh[2], g_prof.evh[3]);
    hb[0] += ti;
    hb[1] += tf;
    hb[5] += 1;
    hb[9] += 8.0 * tri;  // L rows read (an upper bound: zero rows read fewer), A's lower triangle written
    return LDLT_OK;
}

cudaError_t build_graph(const Plan &c, cudaGraphExec_t *exec)
{
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (err != cudaSuccess) return err;
    err = cudaGraphCreate(&g, 0);
    auto fail = [&](cudaError_t e2) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs, &junk);
        }
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        return e2;
    };
    if (err != cudaSuccess) return fail(err);
    // start: status, ingest, loop state
    err = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (err != cudaSuccess) return fail(err);
    err = enqueue_start(c, cs);
    if (err != cudaSuccess) return fail(err);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    err = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (err != cudaSuccess) return fail(err);
    cudaGraphNode_t dep[8];
    if (ndeps > 8) return fail(cudaErrorUnknown);
    for (size_t i = 0; i < ndeps; ++i) dep[i] = deps[i];
    cudaGraph_t tmp = nullptr;
    err = cudaStreamEndCapture(cs, &tmp);
    if (err != cudaSuccess) return fail(err);
    // the panel loop: a while node, condition set by the second half's loop step
    cudaGraphConditionalHandle cond;
    err = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (err != cudaSuccess) return fail(err);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    err = cudaGraphAddNode(&loop, g, dep, nullptr, ndeps, &cp);
    if (err != cudaSuccess) return fail(err);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    err = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (err != cudaSuccess) return fail(err);
    err = enqueue_step(c, 0, cond, 0, nullptr, cs);
    if (err == cudaSuccess) err = enqueue_step(c, 1, cond, 1, nullptr, cs);
    if (err != cudaSuccess) return fail(err);
    err = cudaStreamEndCapture(cs, &tmp);
    if (err != cudaSuccess) return fail(err);
    // finish: L in perm order, D, perm, e, rank
    err = cudaStreamBeginCaptureToGraph(cs, g, &loop, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (err != cudaSuccess) return fail(err);
    err = enqueue_finish(c, cs);
    if (err != cudaSuccess) return fail(err);
    err = cudaStreamEndCapture(cs, &tmp);
    if (err != cudaSuccess) return fail(err);
    err = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    g = nullptr;
    cudaStreamDestroy(cs);
    return err;
}

// Instantiated graphs by their launch arguments (every pointer and size the
// kernels are given), least recently used first out.  Each entry keeps an
// event recorded after its last launch: an entry is destroyed only after
// that launch has finished.
struct GraphKey {
    int64_t n, lda;
    uint32_t p;
    int path, dev, nsm, npend, test_drop;
    int64_t budget;
    const void *A, *perm, *e, *rank, *status, *ws, *gperm, *gbad;
};
struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    uint64_t used = 0;
};
constexpr int GRAPH_CACHE = 4;
std::mutex g_graph_mu;
GraphEntry g_graphs[GRAPH_CACHE];
uint64_t g_graph_clock = 0;

int run_graph(const Plan &c, cudaStream_t st)
{
    GraphKey k;
    std::memset(&k, 0, sizeof(k));
    k.n = c.n; k.lda = c.lda; k.p = c.p; k.path = c.path; k.nsm = c.nsm;
    k.npend = g_npend; k.test_drop = g_test_drop; k.budget = g_budget_ns;
    CK(cudaGetDevice(&k.dev));
    k.A = c.A; k.perm = c.perm; k.e = c.e; k.rank = c.rank; k.status = c.status;
    k.ws = c.Sbuf[0]; k.gperm = c.gperm; k.gbad = c.gbad;
    std::lock_guard<std::mutex> lock(g_graph_mu);
    GraphEntry *hit = nullptr, *lru = &g_graphs[0];
    for (GraphEntry &ge : g_graphs) {
        if (ge.exec && std::memcmp(&ge.key, &k, sizeof(k)) == 0) { hit = &ge; break; }
        if (!ge.exec || (lru->exec && ge.used < lru->used)) lru = &ge;
    }
    if (!hit) {
        cudaGraphExec_t ex = nullptr;
        CK(build_graph(c, &ex));
        if (lru->exec) {
            cudaEventSynchronize(lru->done);  // its last launch has finished
            cudaGraphExecDestroy(lru->exec);
            lru->exec = nullptr;
        }
        if (!lru->done && cudaEventCreateWithFlags(&lru->done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGraphExecDestroy(ex);
            return LDLT_ERR_CUDA;
        }
        std::memcpy(&lru->key, &k, sizeof(k));
        lru->exec = ex;
        hit = lru;
    }
    hit->used = ++g_graph_clock;
    CK(cudaGraphLaunch(hit->exec, st));
    CK(cudaEventRecord(hit->done, st));
    return LDLT_OK;
}

}  // namespace

int factor_core(int64_t n, uint32_t p, uint32_t *A, int64_t lda, int32_t *perm, uint32_t *e, int64_t *rank,
                int32_t *status, int path, void *ws, size_t ws_bytes, void *stream, const int32_t *gperm,
                int *gbad)
{
    int rc = check_args(n, p, path);
    if (rc != LDLT_OK) return rc;
    if (!rank || !status) return LDLT_ERR_ARG;
    if (n > 0 && (!A || !perm || !e || lda < n)) return LDLT_ERR_ARG;
    Layout Lo;
    make_layout(n, p, path, Lo);
    if (!ws || ws_bytes < Lo.total) return LDLT_ERR_WORKSPACE;
    if (((uintptr_t)ws & 255) != 0) return LDLT_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;

    int dev = 0, major = 0, minor = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (major != 10 || minor != 3) return LDLT_ERR_NO_DEVICE;

    if (n == 0) {
        CK(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
        CK(cudaMemsetAsync(rank, 0, sizeof(int64_t), st));
        return LDLT_OK;
    }

    Plan pl;
    plan_make(pl, n, p, path, A, lda, perm, e, rank, status, ws, gperm, gbad, Lo, nsm);
    if (g_prof.on) return run_profiled(pl, st);
    return run_graph(pl, st);
}

extern "C" int rpm_from_factor(int64_t n, const int32_t *perm, const uint32_t *e, const int64_t *rank,
                               int32_t *rpm_col, void *stream)
{
    if (n < 0) return LDLT_ERR_ARG;
    if (n > 0 && (!perm || !e || !rank || !rpm_col)) return LDLT_ERR_ARG;
    CK(launch_rpm(n, perm, e, rank, rpm_col, (cudaStream_t)stream));
    return LDLT_OK;
}
