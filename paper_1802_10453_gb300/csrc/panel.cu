// panel.cu -- the pivot chain: one panel of the lexicographic elimination.
//
// Dumas & Pernet, Algorithm 4 (Section 5).  Rows of the current Schur
// complement S are visited in ascending order.  Row a becomes
//   * a 1x1 pivot if its diagonal entry c_a[a] is non-zero;
//   * a 2x2 pivot with b, the first index > a with c_a[b] != 0;
//   * a non-pivot row if its Schur row is zero.
// c_a[t] = S[t][a] - sum_k Lp[t][k] (D Lp[a])_k is the Crout form of the Schur
// entry (the "c <- A_{i..n,i} - N v^T" step of Algorithm 4, with D in place of
// the printed D^{-1}); Lp holds the L columns of the pivots taken so far in
// this panel.  After a 1x1 pivot the new column is c_a / d; after a 2x2 pivot
// the columns of a and b are alpha_t = (c_b[t] - delta beta_t)/x and
// beta_t = c_a[t]/x (Algorithm 4, 2x2 branch: delta = y/2 for odd p, y for p = 2).
//
// GPU organisation.  One cooperative launch per panel.  CTA 0 (the leader)
// owns the window of the first W rows of S and takes every decision.  The
// other CTAs (helpers) own the far rows [W, m) in contiguous slices; they
// compute the new L columns of their rows as the leader publishes pivots
// (an ordered event queue in global memory), and answer "far scans": when a
// row has no non-zero inside the window, every helper searches its slice for
// the first non-zero of that row and the leader takes the minimum.  Helpers
// never block the leader except during a far scan.  Every wait is bounded by
// a %globaltimer budget; when it runs out the kernel writes LDLT_ERR_TIMEOUT
// to the status word, raises an abort flag the other CTAs poll, and returns.
//
// At the end the leader compacts the remaining rows (order preserved) into
// sigma / idx_next for the next Schur complement.
#include <climits>

#include "ldlt_internal.cuh"

#define LDLT_ERR_TIMEOUT_CODE (-6)

namespace {

__device__ __forceinline__ int64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (int64_t)t;
}

__device__ __forceinline__ uint32_t s_at(const uint32_t *__restrict__ S, int64_t ldS, int i, int j)
{
    return i >= j ? __ldg(S + (int64_t)i * ldS + j) : __ldg(S + (int64_t)j * ldS + i);
}

// sum over the CTA of values < 2^32 (at most 2^10 of them)
__device__ uint64_t block_sum(uint64_t v, uint64_t *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    uint64_t s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__device__ int block_min(int v, int *redi)
{
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) redi[w] = v;
    __syncthreads();
    int s = INT_MAX;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = min(s, redi[i]);
    return s;
}

// (D l)_k for the block diagonal D of this panel (eval[k] != 0 marks the start
// of a 2x2 block [[0,x],[x,dval[k+1]]]).
__device__ __forceinline__ uint32_t dmul(int k, const uint32_t *l, const uint32_t *dval,
                                         const uint32_t *eval, const FieldP &f)
{
    if (eval[k] != 0) return fp_mul(eval[k], l[k + 1], f);
    if (k > 0 && eval[k - 1] != 0)
        return fp_add(fp_mul(eval[k - 1], l[k - 1], f), fp_mul(dval[k], l[k], f), f);
    return fp_mul(dval[k], l[k], f);
}

// c_v[t] = S(t, a) - sum_{k < np} Lp[t][k] v[k]
__device__ __forceinline__ uint32_t schur_entry(const PanelParams &P, int t, int a,
                                                const uint32_t *v, int np)
{
    uint64_t acc = 0;
    const uint32_t *col = P.LpT + t;
    int k = 0;
    for (; k + 4 <= np; k += 4) {
        uint32_t l0 = col[(int64_t)(k + 0) * P.ldL];
        uint32_t l1 = col[(int64_t)(k + 1) * P.ldL];
        uint32_t l2 = col[(int64_t)(k + 2) * P.ldL];
        uint32_t l3 = col[(int64_t)(k + 3) * P.ldL];
        fp_mac(acc, l0, v[k + 0], P.f);
        fp_mac(acc, l1, v[k + 1], P.f);
        fp_mac(acc, l2, v[k + 2], P.f);
        fp_mac(acc, l3, v[k + 3], P.f);
    }
    for (; k < np; ++k) fp_mac(acc, col[(int64_t)k * P.ldL], v[k], P.f);
    return fp_sub(s_at(P.S, P.ldS, t, a), fp_reduce64(acc, P.f), P.f);
}

__device__ void raise_timeout(const PanelParams &P)
{
    atomicExch(P.status, LDLT_ERR_TIMEOUT_CODE);
    atomicExch(&P.sync->abort, 1);
}

// ---------------------------------------------------------------------------
// helper CTAs
// ---------------------------------------------------------------------------
__device__ void helper_loop(const PanelParams &P, int lo, int hi)
{
    __shared__ uint32_t sv_a[KP_MAX], sv_b[KP_MAX];
    __shared__ Event ev;
    __shared__ int s_go;
    __shared__ int redi[32];
    const int tid = threadIdx.x;
    const int cta = blockIdx.x;
    for (int e = 0;; ++e) {
        if (tid == 0) {
            int go = 0;
            int64_t t0 = gtime();
            volatile int *cnt = &P.sync->ev_count;
            volatile int *ab = &P.sync->abort;
            for (;;) {
                if (*cnt > e) { go = 1; break; }
                if (*ab) break;
                if (gtime() - t0 > P.budget_ns) { raise_timeout(P); break; }
            }
            __threadfence();
            if (go) {
                ev.kind = __ldcg(&P.events[e].kind);
                ev.a = __ldcg(&P.events[e].a);
                ev.b = __ldcg(&P.events[e].b);
                ev.np = __ldcg(&P.events[e].np);
                ev.s0 = __ldcg(&P.events[e].s0);
                ev.s1 = __ldcg(&P.events[e].s1);
                ev.scan_id = __ldcg(&P.events[e].scan_id);
            }
            s_go = go;
        }
        __syncthreads();
        if (!s_go || ev.kind == EV_END) return;
        const int np = ev.np, a = ev.a, b = ev.b, kind = ev.kind;
        const uint32_t *vv = P.evvec + (int64_t)e * 2 * KP_MAX;
        for (int k = tid; k < np; k += blockDim.x) {
            sv_a[k] = __ldcg(vv + k);
            if (kind == EV_PIVOT2) sv_b[k] = __ldcg(vv + KP_MAX + k);
        }
        __syncthreads();
        int firstnz = INT_MAX;
        for (int t = lo + tid; t < hi; t += blockDim.x) {
            if (kind == EV_PIVOT1) {
                uint32_t c = schur_entry(P, t, a, sv_a, np);
                P.LpT[(int64_t)np * P.ldL + t] = fp_mul(c, ev.s0, P.f);
            } else if (kind == EV_PIVOT2) {
                uint32_t ca = schur_entry(P, t, a, sv_a, np);
                uint32_t cb = schur_entry(P, t, b, sv_b, np);
                uint32_t beta = fp_mul(ca, ev.s0, P.f);
                uint32_t alpha = fp_mul(fp_sub(cb, fp_mul(beta, ev.s1, P.f), P.f), ev.s0, P.f);
                P.LpT[(int64_t)np * P.ldL + t] = alpha;
                P.LpT[(int64_t)(np + 1) * P.ldL + t] = beta;
            } else {  // EV_SCAN
                uint32_t c = schur_entry(P, t, a, sv_a, np);
                if (c != 0 && t < firstnz) firstnz = t;
            }
        }
        if (kind == EV_SCAN) {
            int mn = block_min(firstnz, redi);
            if (mn != INT_MAX) {
                for (int k = tid; k < np; k += blockDim.x)
                    P.partner_lp[(int64_t)cta * KP_MAX + k] = P.LpT[(int64_t)k * P.ldL + mn];
            }
            if (tid == 0) P.scan_min[cta] = mn;
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicAdd(&P.sync->scan_done, 1);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// leader CTA
// ---------------------------------------------------------------------------
struct LeaderShared {
    uint32_t va[KP_MAX], vb[KP_MAX], la[KP_MAX], lb[KP_MAX];
    uint32_t dval[KP_MAX], eval[KP_MAX];
    int piv_rows[KP_MAX];
    int zero_rows[W0];
    int zero_np[W0];
    uint8_t wstate[W0];
    uint64_t red[32];
    int redi[32];
    int np, ia, nzero, nev, nscan, b, abort;
    uint32_t x, y;
};

__device__ void publish(const PanelParams &P, LeaderShared &sh, int kind, int a, int b, int np,
                        uint32_t s0, uint32_t s1, int scan_id)
{
    const int tid = threadIdx.x;
    const int e = sh.nev;
    uint32_t *vv = P.evvec + (int64_t)e * 2 * KP_MAX;
    for (int k = tid; k < np; k += blockDim.x) {
        vv[k] = sh.va[k];
        if (kind == EV_PIVOT2) vv[KP_MAX + k] = sh.vb[k];
    }
    if (tid == 0) {
        Event *ev = &P.events[e];
        ev->kind = kind; ev->a = a; ev->b = b; ev->np = np;
        ev->s0 = s0; ev->s1 = s1; ev->scan_id = scan_id; ev->pad = 0;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        atomicExch(&P.sync->ev_count, e + 1);
        sh.nev = e + 1;
    }
    __syncthreads();
}

__device__ void leader_loop(const PanelParams &P, bool helpers)
{
    __shared__ LeaderShared sh;
    const int tid = threadIdx.x;
    const FieldP f = P.f;
    const int w = P.w;
    for (int t = tid; t < W0; t += blockDim.x) sh.wstate[t] = 0;
    if (tid == 0) {
        sh.np = 0; sh.ia = 0; sh.nzero = 0; sh.nev = 0; sh.nscan = 0; sh.abort = 0;
    }
    __syncthreads();

    for (;;) {
        const int np = sh.np, ia = sh.ia;
        if (np > P.kp - 2 || ia >= w || sh.abort) break;
        if (sh.wstate[ia]) {
            __syncthreads();
            if (tid == 0) sh.ia = ia + 1;
            __syncthreads();
            continue;
        }
        const int a = ia;
        // L row of a over this panel's columns, then v_a = D l_a
        for (int k = tid; k < np; k += blockDim.x) sh.la[k] = P.LpT[(int64_t)k * P.ldL + a];
        __syncthreads();
        for (int k = tid; k < np; k += blockDim.x) sh.va[k] = dmul(k, sh.la, sh.dval, sh.eval, f);
        __syncthreads();
        uint64_t part = 0;
        for (int k = tid; k < np; k += blockDim.x) part += fp_mul(sh.la[k], sh.va[k], f);
        uint32_t caa = fp_sub(s_at(P.S, P.ldS, a, a), fp_reduce64(block_sum(part, sh.red), f), f);

        if (caa != 0) {
            // ---- 1x1 pivot ----
            uint32_t dinv = fp_inv(caa, f);
            if (helpers) publish(P, sh, EV_PIVOT1, a, -1, np, dinv, 0, 0);
            {
                const int t = tid;  // window rows: one per thread (w <= W0 == blockDim.x)
                if (t >= a && t < w) {
                    uint32_t c = schur_entry(P, t, a, sh.va, np);
                    P.LpT[(int64_t)np * P.ldL + t] = fp_mul(c, dinv, f);
                }
            }
            __syncthreads();
            if (tid == 0) {
                sh.piv_rows[np] = a; sh.dval[np] = caa; sh.eval[np] = 0;
                sh.wstate[a] = 1; sh.np = np + 1; sh.ia = ia + 1;
            }
            __syncthreads();
            continue;
        }

        // ---- first non-zero of row a beyond a, inside the window ----
        uint32_t ca_t = 0;  // c_a[t] for the thread's window row t (one row per thread)
        int firstnz = INT_MAX;
        {
            const int t = tid;
            if (t > a && t < w) {
                ca_t = schur_entry(P, t, a, sh.va, np);
                if (ca_t != 0) firstnz = t;
            }
        }
        int b = block_min(firstnz, sh.redi);
        bool far = false;
        if (b == INT_MAX && helpers) {
            // ---- far scan over the helpers' rows ----
            const int scan_id = sh.nscan;
            publish(P, sh, EV_SCAN, a, -1, np, 0, 0, scan_id);
            if (tid == 0) {
                const int target = (scan_id + 1) * (int)(gridDim.x - 1);
                volatile int *done = &P.sync->scan_done;
                volatile int *ab = &P.sync->abort;
                int64_t t0 = gtime();
                int ok = 0;
                for (;;) {
                    if (*done >= target) { ok = 1; break; }
                    if (*ab) break;
                    if (gtime() - t0 > P.budget_ns) { raise_timeout(P); break; }
                }
                __threadfence();
                int best = INT_MAX, owner = -1;
                if (ok) {
                    for (int c = 1; c < (int)gridDim.x; ++c) {
                        int v = __ldcg(&P.scan_min[c]);
                        if (v < best) { best = v; owner = c; }
                    }
                } else {
                    sh.abort = 1;
                }
                sh.b = best;
                sh.redi[0] = owner;
                sh.nscan = scan_id + 1;
            }
            __syncthreads();
            if (sh.abort) break;
            b = sh.b;
            const int owner = sh.redi[0];
            if (b != INT_MAX) {
                far = true;
                for (int k = tid; k < np; k += blockDim.x)
                    sh.lb[k] = __ldcg(&P.partner_lp[(int64_t)owner * KP_MAX + k]);
            }
            __syncthreads();
        }
        if (b == INT_MAX) {
            // ---- zero row ----
            __syncthreads();
            if (tid == 0) {
                sh.zero_rows[sh.nzero] = a; sh.zero_np[sh.nzero] = np; sh.nzero += 1;
                sh.wstate[a] = 1; sh.ia = ia + 1;
            }
            __syncthreads();
            continue;
        }

        // ---- 2x2 pivot on (a, b) ----
        if (!far)
            for (int k = tid; k < np; k += blockDim.x) sh.lb[k] = P.LpT[(int64_t)k * P.ldL + b];
        __syncthreads();
        for (int k = tid; k < np; k += blockDim.x) sh.vb[k] = dmul(k, sh.lb, sh.dval, sh.eval, f);
        __syncthreads();
        uint64_t px = 0, py = 0;
        for (int k = tid; k < np; k += blockDim.x) {
            px += fp_mul(sh.lb[k], sh.va[k], f);
            py += fp_mul(sh.lb[k], sh.vb[k], f);
        }
        uint32_t x = fp_sub(s_at(P.S, P.ldS, a, b), fp_reduce64(block_sum(px, sh.red), f), f);
        uint32_t y = fp_sub(s_at(P.S, P.ldS, b, b), fp_reduce64(block_sum(py, sh.red), f), f);
        uint32_t xinv = fp_inv(x, f);
        uint32_t delta = (f.p == 2) ? y : fp_mul(y, f.inv2, f);
        if (helpers) publish(P, sh, EV_PIVOT2, a, b, np, xinv, delta, 0);
        {
            const int t = tid;
            if (t >= a && t < w) {
            const uint32_t ca = (t == a) ? 0u : ca_t;  // c_a[a] = 0 (no 1x1 pivot)
            uint32_t cb = schur_entry(P, t, b, sh.vb, np);
            uint32_t beta = fp_mul(ca, xinv, f);
            uint32_t alpha = fp_mul(fp_sub(cb, fp_mul(beta, delta, f), f), xinv, f);
            P.LpT[(int64_t)np * P.ldL + t] = alpha;
            P.LpT[(int64_t)(np + 1) * P.ldL + t] = beta;
            }
        }
        __syncthreads();
        if (tid == 0) {
            sh.piv_rows[np] = a; sh.piv_rows[np + 1] = b;
            sh.dval[np] = 0; sh.dval[np + 1] = (f.p == 2) ? y : 0;
            sh.eval[np] = x; sh.eval[np + 1] = 0;
            sh.wstate[a] = 1;
            if (b < w) sh.wstate[b] = 1;
            P.consumed[b] = 1;
            sh.np = np + 2; sh.ia = ia + 1;
        }
        __syncthreads();
    }

    if (helpers && !sh.abort) publish(P, sh, EV_END, -1, -1, 0, 0, 0, 0);
    __threadfence();
    __syncthreads();

    // ---- report ----
    const int np = sh.np, iend = sh.ia, nzero = sh.nzero;
    for (int k = tid; k < np; k += blockDim.x) {
        P.out->piv_rows[k] = sh.piv_rows[k];
        P.out->dval[k] = sh.dval[k];
        P.out->eval[k] = sh.eval[k];
    }
    for (int q = tid; q < nzero; q += blockDim.x) {
        P.out->zero_rows[q] = sh.zero_rows[q];
        P.out->zero_np[q] = sh.zero_np[q];
    }

    // ---- compaction of the remaining rows [iend, m) minus consumed partners ----
    const int m = P.m;
    const int len = m - iend;
    const int per = (len + blockDim.x - 1) / blockDim.x;
    const int lo = iend + tid * per, hi = min(m, lo + per);
    int cnt = 0;
    for (int t = lo; t < hi; ++t) cnt += P.consumed[t] ? 0 : 1;
    // exclusive scan of cnt over the CTA
    int incl = cnt;
    const int lane = tid & 31, wid = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    __syncthreads();
    if (lane == 31) sh.redi[wid] = incl;
    __syncthreads();
    int woff = 0, total = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
        if (i < wid) woff += sh.redi[i];
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
    }
}

__global__ void __launch_bounds__(PANEL_THREADS) panel_kernel(PanelParams P)
{
    const bool helpers = gridDim.x > 1;
    if (blockIdx.x == 0) {
        leader_loop(P, helpers);
    } else {
        const int nh = gridDim.x - 1;
        const int far = P.m - P.w;
        const int chunk = (far + nh - 1) / nh;
        const int lo = P.w + (blockIdx.x - 1) * chunk;
        const int hi = min(P.m, lo + chunk);
        helper_loop(P, lo, hi);
    }
}

}  // namespace

cudaError_t launch_panel(const PanelParams &pp, int grid, cudaStream_t st)
{
    PanelParams p = pp;
    void *args[] = {&p};
    if (grid <= 1)
        return cudaLaunchKernel((const void *)panel_kernel, dim3(1), dim3(PANEL_THREADS), args, 0, st);
    return cudaLaunchCooperativeKernel((const void *)panel_kernel, dim3(grid), dim3(PANEL_THREADS),
                                       args, 0, st);
}
