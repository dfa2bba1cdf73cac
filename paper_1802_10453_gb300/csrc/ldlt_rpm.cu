// ldlt_rpm.cu -- host side of the C ABI declared in include/ldlt_rpm.h.
//
// Blocked right-looking form of the lexicographic elimination (Algorithm 4's
// pivot order, Algorithm 2's level-3 updates):
//   ingest:   S = lower(A) mod p, compact index = original index
//   repeat:   panel   -- pivot chain over the first W0 rows of S (panel.cu):
//                        up to KP_MAX pivots, their L columns for every row
//             record  -- append pivots / D / zero rows to the global lists
//             store   -- L columns into Lw (by original row)
//             update  -- S <- S[sigma, sigma] - G D G^T on the remaining rows
//                        (SYRDK, FP64 or tensor-core form), rows compacted
//   finalize: A <- L in perm order with D on the diagonal (PERM)
// After each panel three words are read back to size the next launches.
#include <cstddef>
#include <cstdio>
#include <cstring>

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
    cudaEvent_t evs[2][4] = {};  // two sets: panel i uses set i & 1
    int pending = -1;            // set whose events are recorded but not yet read
    bool ready = false;
};
Prof g_prof;

void prof_init()
{
    if (!g_prof.ready) {
        for (auto &s : g_prof.evs)
            for (auto &e : s) cudaEventCreate(&e);
        g_prof.ready = true;
    }
}

// Accumulate the phase times of the last recorded panel (its events have
// completed: the caller synchronised the stream after them).
void prof_collect()
{
    if (g_prof.pending < 0) return;
    cudaEvent_t *ev = g_prof.evs[g_prof.pending];
    cudaEventSynchronize(ev[3]);
    float t01 = 0, t12 = 0, t23 = 0;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    g_prof.acc[0] += t01;
    g_prof.acc[1] += t12;
    g_prof.acc[2] += t23;
    g_prof.pending = -1;
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
    size_t out, sync, evlog, scans, partner_lp, scancol, zlog, opA, opB, total;
};

constexpr int MAX_GRID = 1024;

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
    g_prof.pending = -1;
}

extern "C" int ldlt_rpm_profile_read(double out[32])
{
    if (!out) return LDLT_ERR_ARG;
    prof_collect();
    for (int i = 0; i < 32; ++i) out[i] = g_prof.acc[i];
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

    CK(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    if (n == 0) {
        CK(cudaMemsetAsync(rank, 0, sizeof(int64_t), st));
        return LDLT_OK;
    }

    uint8_t *w = (uint8_t *)ws;
    uint32_t *Sbuf[2] = {(uint32_t *)(w + Lo.S0), (uint32_t *)(w + Lo.S1)};
    uint32_t *Lw = (uint32_t *)(w + Lo.Lw);
    uint32_t *LpT = (uint32_t *)(w + Lo.LpT);
    uint32_t *LpC = (uint32_t *)(w + Lo.LpC);
    int *idxb[2] = {(int *)(w + Lo.idx0), (int *)(w + Lo.idx1)};
    int *sigma = (int *)(w + Lo.sigma);
    uint8_t *consumed = w + Lo.consumed;
    int *piv_all = (int *)(w + Lo.piv_all);
    uint32_t *d_all = (uint32_t *)(w + Lo.d_all);
    uint32_t *e_all = (uint32_t *)(w + Lo.e_all);
    int *zero_all = (int *)(w + Lo.zero_all);
    int *zero_cols = (int *)(w + Lo.zero_cols);
    PanelOut *out = (PanelOut *)(w + Lo.out);
    PanelSync *sync = (PanelSync *)(w + Lo.sync);
    const int64_t ldS = Lo.ldS;
    const FieldP f = make_field(p);
    const int limbs = (path == LDLT_PATH_TC) ? tc_limbs(p) : 0;

    if (gperm) CK(launch_ingest_perm(A, lda, n, gperm, Sbuf[0], ldS, idxb[0], f, gbad, st));
    else CK(launch_ingest(A, lda, n, Sbuf[0], ldS, idxb[0], f, st));
    const bool prof = g_prof.on;
    if (prof) g_prof.acc[5] += 1;

    int m = (int)n, r0 = 0, z0 = 0, cur = 0, ipanel = 0;
    while (m > 0) {
        cudaEvent_t *ev = g_prof.evs[ipanel & 1];
        CK(cudaMemset2DAsync(LpT, (size_t)ldS * 4, 0, (size_t)m * 4, KP_MAX, st));
        CK(cudaMemsetAsync(consumed, 0, (size_t)m, st));
        CK(cudaMemsetAsync(sync, 0, sizeof(PanelSync), st));

        PanelParams pp;
        pp.S = Sbuf[cur]; pp.ldS = ldS; pp.m = m; pp.f = f;
        pp.kp = KP_MAX; pp.w = m < W0 ? m : W0;
        pp.LpT = LpT; pp.LpC = LpC; pp.ldL = ldS;
        pp.consumed = consumed; pp.idx = idxb[cur]; pp.sigma = sigma; pp.idx_next = idxb[cur ^ 1];
        pp.out = out; pp.sync = sync;
        pp.evlog = (uint32_t *)(w + Lo.evlog);
        pp.scans = (ScanSlot *)(w + Lo.scans); pp.partner_lp = (uint32_t *)(w + Lo.partner_lp);
        pp.scancol = (uint32_t *)(w + Lo.scancol);
        pp.zlog = (uint32_t *)(w + Lo.zlog);
        pp.budget_ns = g_budget_ns; pp.status = status;
        pp.npend = g_npend;
        pp.test_drop = g_test_drop;
        int grid = 1;
        if (m > pp.w) {
            // spread the far rows over every SM, at least MIN_HELPER_ROWS rows per helper
            const int need = 1 + (m - pp.w + MIN_HELPER_ROWS - 1) / MIN_HELPER_ROWS;
            grid = need < nsm ? need : nsm;
            if (grid > MAX_PANEL_GRID) grid = MAX_PANEL_GRID;
        }
        if (prof) CK(cudaEventRecord(ev[0], st));
        CK(launch_panel(pp, grid, st));
        CK(launch_record_panel(out, idxb[cur], r0, z0, piv_all, d_all, e_all, zero_all, zero_cols, st));
        struct { int h[8]; long long cyc[8]; long long dbg[16]; } rb;
        static_assert(offsetof(PanelOut, cyc) == 8 * sizeof(int), "PanelOut layout");
        CK(cudaMemcpyAsync(&rb, out, sizeof(rb), cudaMemcpyDeviceToHost, st));
        const int *hdr = rb.h;
        if (prof) CK(cudaEventRecord(ev[1], st));
        CK(cudaStreamSynchronize(st));
        if (prof) prof_collect();  // the previous panel's events precede this sync
        const int np = hdr[0], nzero = hdr[1], m_next = hdr[3], aborted = hdr[4];
        if (prof) {
            g_prof.acc[5] += 2;  // panel, record
            g_prof.acc[6] += 1;
            g_prof.acc[7] += hdr[5];
            for (int i = 0; i < 8; ++i) g_prof.acc[8 + i] += (double)rb.cyc[i];
            for (int i = 0; i < 16; ++i) g_prof.acc[16 + i] += (double)rb.dbg[i];
        }
        if (aborted) return LDLT_OK;  // LDLT_ERR_TIMEOUT is in *status
        CK(launch_lw_scatter(LpC, ldS, m, np, idxb[cur], Lw, ldS, r0, st));
        if (prof && np > 0) g_prof.acc[5] += 1;
        bool upd = false;
        if (m_next > 0) {
            if (np > 0) {
                const int kpad = (int)round_up(np, 64);
                if (path == LDLT_PATH_FP64) {
                    double *GDT = (double *)(w + Lo.opA);
                    double *GT = GDT + (size_t)KP_MAX * ldS;
                    CK(launch_split_fp64(LpC, ldS, sigma, m_next, np, out, f, GDT, GT, ldS, kpad, st));
                    if (prof) CK(cudaEventRecord(ev[2], st));
                    upd = true;
                    CK(launch_syrdk_fp64(Sbuf[cur], ldS, sigma, m_next, GDT, GT, ldS, kpad, f,
                                         Sbuf[cur ^ 1], st));
                } else {
                    uint8_t *opA = w + Lo.opA;
                    const size_t aBytes = (size_t)round_up(round_up(n, 128) * (int64_t)limbs * KP_MAX * 2, 256);
                    uint8_t *opB = opA + aBytes;
                    CK(launch_split_tc(LpC, ldS, sigma, m_next, np, out, f, limbs, kpad, opA, opB, st));
                    if (prof) CK(cudaEventRecord(ev[2], st));
                    upd = true;
                    CK(launch_syrdk_tc(Sbuf[cur], ldS, sigma, m_next, opA, opB, limbs, kpad, f,
                                       Sbuf[cur ^ 1], g_budget_ns, status, nsm,
                                       g_test_drop == LDLT_TEST_DROP_UPDATE_COPIES, st));
                }
            } else {
                CK(launch_compact_copy(Sbuf[cur], ldS, sigma, m_next, Sbuf[cur ^ 1], st));
                if (prof) g_prof.acc[5] += 1;
            }
        }
        if (prof) {
            if (!upd) CK(cudaEventRecord(ev[2], st));
            CK(cudaEventRecord(ev[3], st));
            g_prof.pending = ipanel & 1;
            if (upd) {
                g_prof.acc[3] += (double)m_next * (double)(m_next + 1) * 0.5 * (double)np;
                g_prof.acc[4] += 1;
                g_prof.acc[5] += 2;  // split, update
            }
        }
        r0 += np;
        z0 += nzero;
        cur ^= 1;
        m = m_next;
        ++ipanel;
    }
    CK(launch_finalize(n, Lw, ldS, piv_all, d_all, e_all, zero_all, zero_cols, r0, A, lda, perm, e, rank, st));
    if (prof) g_prof.acc[5] += 1;
    return LDLT_OK;
}

extern "C" int rpm_from_factor(int64_t n, const int32_t *perm, const uint32_t *e, const int64_t *rank,
                               int32_t *rpm_col, void *stream)
{
    if (n < 0) return LDLT_ERR_ARG;
    if (n > 0 && (!perm || !e || !rank || !rpm_col)) return LDLT_ERR_ARG;
    CK(launch_rpm(n, perm, e, rank, rpm_col, (cudaStream_t)stream));
    return LDLT_OK;
}
