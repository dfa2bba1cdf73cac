// ldlt_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "field.cuh"

// Panel geometry.  A panel takes at most KP_MAX pivots (L columns) from the
// window of the first W0 remaining rows; its far rows are shared by helper CTAs.
constexpr int KP_MAX = 128;
constexpr int W0 = 256;
constexpr int ROWS_PER_HELPER = 256;  // far rows per helper CTA kept in shared memory
constexpr int MIN_HELPER_ROWS = 64;   // fewer rows than this per helper is not worth a CTA
constexpr int PANEL_THREADS_V2 = 576; // 16 compute warps (two threads per row) + 2 service warps
constexpr int MAX_EVENTS = 8192;      // events per panel (a panel ends early at the cap)
constexpr int MAX_SCANS = 4096;       // far scans per panel (re-issued scans included)
constexpr int SCAN_RING = 64;         // per-scan buffers (candidate rows, scan columns), by scan id
constexpr int PSTR = KP_MAX + 8;      // words per candidate row: U~ values, then x~ at KP_MAX
constexpr int ZLOG_EV = 64;           // recent row events whose z vectors the leader keeps
constexpr int MAX_PANEL_GRID = 256;
constexpr int EV_WORDS = 4 * KP_MAX;  // payload words per event
constexpr int EV_REC = 8 + EV_WORDS;  // event record: header (one Event) then payload

// Row storage of the Schur complement and of L: leading dimension rounded up so
// every row starts on a 256-byte boundary.
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

enum EventKind : int { EV_PIVOT1 = 1, EV_PIVOT2 = 2, EV_SCAN = 3, EV_END = 4 };

// One message from the leader CTA to the helper CTAs (see panel.cu).
struct Event {
    int kind;
    int a, b;        // compact rows of the pivot (b only for 2x2)
    int np;          // length of the z vectors (storage columns they cover)
    uint32_t s0;     // the scale W of the division-free Crout form
    int col;         // storage column the event writes (pivots), else -1
    int scan_id;     // EV_SCAN: scan id
    int aux;         // unused (zero)
};

// Counters the CTAs of one panel launch share (zeroed before the launch).
struct PanelSync {
    int ev_count;    // events published by the leader
    int scan_done;   // unused
    int abort;       // set by whoever times out
    int pad;
};

// Answer to one far scan: helpers lower `min` to their first non-zero row and
// then count themselves in `done` (initialised to done = 0, min = INT_MAX).
struct ScanSlot {
    int done;           // helpers that answered
    int min;            // smallest row with a non-zero entry, INT_MAX if none yet
    unsigned mask[8];   // bit h: helper CTA h answered (its min is in above)
    int pad[6];
};
static_assert(MAX_PANEL_GRID <= 8 * 32, "one answer bit per helper CTA");

// What the panel kernel reports to the kernels that follow it.  Pivots, D
// and the L columns (LpC) are in pivot order.
struct PanelOut {
    int np;          // pivots taken in this panel (L columns)
    int nzero;       // non-pivot rows found
    int iend;        // first window row not processed
    int m_next;      // order of the next Schur complement
    int abort;
    int nscan;       // far scans issued, re-issued ones included (diagnostics)
    int pad[2];
    long long cyc[8];       // unused (zero)
    long long dbg[16];      // pivot-chain counters (see ldlt_rpm_profile_read)
    uint32_t dval[KP_MAX];  // D diagonal
    uint32_t eval[KP_MAX];  // x at a 2x2 block start, else 0
};

// State of the panel loop, in device memory: every kernel of a panel step
// reads its sizes here and in PanelOut, so the whole loop is enqueued (a
// CUDA graph with a device-side while condition) without the host reading
// anything back.
struct LoopState {
    int m;           // order of the current Schur complement
    int r0;          // pivots (L columns) taken by earlier panels
    int z0;          // non-pivot rows found by earlier panels
    int done;        // 1 once the factorisation has ended (finished or aborted)
    int aborted;     // 1 if it ended on an error (status holds the code)
    int npanel;      // panels run
    int pad[2];
};

// Helper CTAs a panel over m rows uses, at most `cap` (the launched grid).
__host__ __device__ inline int panel_grid(int m, int cap)
{
    const int w = m < W0 ? m : W0;
    if (m <= w) return 1;
    const int need = 1 + (m - w + MIN_HELPER_ROWS - 1) / MIN_HELPER_ROWS;
    return need < cap ? need : cap;
}

struct PanelParams {
    const uint32_t *S;      // compact Schur complement, lower triangle, ldS
    int64_t ldS;
    const LoopState *ls;    // m = ls->m rows, window min(W0, m)
    FieldP f;
    int kp;                 // pivot budget of this panel (<= KP_MAX)
    uint32_t *LpT;          // LpT[k * ldL + t]: scaled Schur column k (storage order) of compact row t,
                            // for helper rows beyond the CTA's shared memory only
    uint32_t *LpC;          // LpC[k * ldL + t]: L entry of compact row t, pivot-order column k (output)
    int64_t ldL;
    uint8_t *consumed;      // [m]: partner rows taken by 2x2 pivots (zeroed)
    const int *idx;         // [m]: original index of compact row
    int *sigma;             // [m]: out, new compact row -> old compact row
    int *idx_next;          // [m]: out, original index of new compact row
    PanelOut *out;
    PanelSync *sync;
    // the factorisation's lists, appended at ls->r0 / ls->z0 (original indices)
    int *piv_all;           // pivot rows, pivot order
    uint32_t *d_all;        // D
    uint32_t *e_all;        // x at a 2x2 block start, else 0
    int *zero_all;          // non-pivot rows
    int *zero_cols;         // L columns that existed when each was found zero
    uint32_t *evlog;        // [MAX_EVENTS][EV_REC] event records
    ScanSlot *scans;        // [MAX_SCANS]
    uint32_t *partner_lp;   // [SCAN_RING][MAX_PANEL_GRID][PSTR]: candidate rows per scan
    uint32_t *scancol;      // [SCAN_RING][ldL]: scaled far values of each scan's row
    uint32_t *zlog;         // [ZLOG_EV][2][KP_MAX]: z vectors of the leader's recent row events
    int64_t budget_ns;
    int32_t *status;
    int npend;              // far scans allowed in flight (1..16)
    int test_drop;          // LDLT_TEST_DROP_SCAN_ANSWERS: helpers never answer a far scan
};

// ---- launchers (host) -------------------------------------------------------
cudaError_t launch_ingest(const uint32_t *A, int64_t lda, int64_t n, uint32_t *S, int64_t ldS,
                          int *idx, FieldP f, cudaStream_t st);
cudaError_t launch_ingest_perm(const uint32_t *A, int64_t lda, int64_t n, const int32_t *perm, uint32_t *S,
                               int64_t ldS, int *idx, FieldP f, int *bad, cudaStream_t st);
// ldlt_rpm_factor's body; with gperm != NULL it factors P^T A P for that
// order (perm[k] = original index of position k), flagging a bad index in *gbad
int factor_core(int64_t n, uint32_t p, uint32_t *A, int64_t lda, int32_t *perm, uint32_t *e, int64_t *rank,
                int32_t *status, int path, void *ws, size_t ws_bytes, void *stream, const int32_t *gperm,
                int *gbad);
cudaError_t launch_panel(const PanelParams &pp, int grid, cudaStream_t st);
// The per-panel kernels below size themselves from LoopState / PanelOut;
// their grids are fixed for order n and surplus CTAs return at once.
cudaError_t launch_lw_scatter(const uint32_t *LpC, int64_t ldL, int64_t n, const LoopState *ls,
                              const PanelOut *out, const int *idx, uint32_t *Lw, int64_t ldw,
                              cudaStream_t st);
// init != 0: start the loop at order n.  Otherwise advance it past the panel
// in `out` (end it when nothing remains, on an abort, on an error status, or
// if a panel retired no row), and, with set_cond, set the graph's while
// condition to "not done".  Either way the next panel's partner flags
// (consumed) and PanelSync are cleared.
cudaError_t launch_loop_step(LoopState *ls, const PanelOut *out, int init, int64_t n, int32_t *status,
                             uint8_t *consumed, PanelSync *sync, cudaGraphConditionalHandle cond, int set_cond,
                             int num_sms, cudaStream_t st);
cudaError_t launch_finalize(int64_t n, const uint32_t *Lw, int64_t ldw, const int *piv_all,
                            const uint32_t *d_all, const uint32_t *e_all, const int *zero_all,
                            const int *zero_cols, const LoopState *ls, uint32_t *A, int64_t lda,
                            int32_t *perm, uint32_t *e, int64_t *rank, cudaStream_t st);
cudaError_t launch_rpm(int64_t n, const int32_t *perm, const uint32_t *e, const int64_t *rank,
                       int32_t *rpm_col, cudaStream_t st);

// FP64 form of the level-3 update.
size_t fp64_operand_bytes(int64_t n);
// The operand split kernels also do the update of a panel without pivots:
// Snext[i][j] = S[sigma i][sigma j] (rows dropped, nothing subtracted).
cudaError_t launch_split_fp64(const uint32_t *LpC, int64_t ldL, const int *sigma, int64_t n,
                              const LoopState *ls, const PanelOut *out, FieldP f, double *GDT,
                              double *GT, int64_t ldg, const uint32_t *S, int64_t ldS, uint32_t *Snext,
                              cudaStream_t st);
cudaError_t launch_syrdk_fp64(const uint32_t *S, int64_t ldS, const int *sigma, int64_t n,
                              const LoopState *ls, const PanelOut *out, const double *GDT,
                              const double *GT, int64_t ldg, FieldP f, uint32_t *Snext,
                              cudaStream_t st);

// Tensor-core form of the level-3 update.
int tc_limbs(uint32_t p);
int tc_limbs_a(uint32_t p, int *shift);
int tc_bn(int limbs);
size_t tc_operand_bytes(int64_t n, int limbs);
cudaError_t launch_split_tc(const uint32_t *LpC, int64_t ldL, const int *sigma, int64_t n,
                            const LoopState *ls, const PanelOut *out, FieldP f, int limbs,
                            void *Aop, void *Bop, const uint32_t *S, int64_t ldS, uint32_t *Snext,
                            cudaStream_t st);
// upper = 1: the output (i, j), j <= i, is read from and written to S[j][i]
// (TRSS's trailing update of an upper triangle; sigma the identity, S == Snext).
cudaError_t launch_syrdk_tc(const uint32_t *S, int64_t ldS, const int *sigma, const LoopState *ls,
                            const PanelOut *out, const void *Aop, const void *Bop, int limbs,
                            FieldP f, uint32_t *Snext, int64_t budget_ns, int32_t *status,
                            int num_sms, int test_drop, cudaStream_t st, int upper = 0);

// A panel step is live while the loop has not ended and its panel did not
// abort; the kernels after the panel do nothing otherwise.
__device__ __forceinline__ bool step_live(const LoopState *ls, const PanelOut *out)
{
    return !ls->done && !out->abort;
}

// Snext[i][j] = S[sigma i][sigma j], j <= i < m_next, for a panel without
// pivots; CTA b of nb takes rows b, b + nb, ...
__device__ __forceinline__ void compact_rows(const uint32_t *__restrict__ S, int64_t ldS,
                                             const int *__restrict__ sigma, int m_next,
                                             uint32_t *__restrict__ Snext, int b, int nb)
{
    for (int i = b; i < m_next; i += nb) {
        const uint32_t *src = S + (int64_t)sigma[i] * ldS;
        uint32_t *dst = Snext + (int64_t)i * ldS;
        for (int j = threadIdx.x; j <= i; j += blockDim.x) dst[j] = src[sigma[j]];
    }
}
