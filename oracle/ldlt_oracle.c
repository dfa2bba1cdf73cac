/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow CPU restatement of the rank-profile-revealing symmetric
 * factorisation P^T A P = L D L^T over Z/pZ (Dumas & Pernet, "Symmetric
 * indefinite triangular factorization revealing the rank profile matrix",
 * abstract and Section 2; pivoting rule of Algorithm 4, Section 5).
 *
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may
 * load this code.  It shares nothing with the CUDA path: no headers, no
 * helpers, no tables.
 *
 * What it computes.  Rows of the working Schur complement S are visited in
 * ascending original index, skipping rows already consumed as the partner of a
 * 2x2 pivot (Algorithm 4 iterates over rows; after a 2x2 pivot the partner row
 * has been rotated above, so it is never visited again).  For the current row a:
 *
 *   1x1  S_aa != 0                  (Algorithm 4: first non-zero of the row
 *                                    is the diagonal one, j = 0)
 *   2x2  S_aa == 0 and b = the smallest remaining index > a with S_ab != 0
 *                                   (Algorithm 4: "smallest index j such that
 *                                    c_j != 0", j > 0)
 *   none the Schur row is zero      (Algorithm 4: "if c = 0 loop to next
 *                                    iteration"; the row stays a non-pivot row)
 *
 * Algorithm 4 delays the updates (Crout schedule).  Here every pivot updates
 * the whole remaining Schur complement at once (right-looking).  In exact
 * arithmetic both schedules see the same Schur rows, hence take the same pivots
 * and produce the same L and D.
 *
 * 2x2 pivot values (Algorithm 4, 2x2 branch): x = S_ab, y = S_bb,
 *   odd p:  D block [[0,x],[x,0]], y' = y/2, in-block L entry y'/x,
 *   p = 2:  D block [[0,x],[x,y]] (relaxed lower antitriangular block of
 *           Section 2.2), y' = 0, in-block L entry 0;
 *   other rows t: beta_t = S_ta / x (column of b),
 *                 alpha_t = (S_tb - beta_t * delta) / x (column of a),
 *   with delta = y' for odd p and delta = y for p = 2 (the h' update of
 *   Algorithm 4).  The D^{-1} written in the Crout GEMV of Algorithm 4 is read
 *   as D, as Algorithm 2 (G = X^T D^{-1}, Z = C - G D G^T) requires.
 *
 * Output convention (matches the library boundary):
 *   perm[k]  original index of row/column k of P^T A P (pivots in the order
 *            found, a before b for a pair, then the non-pivot rows ascending;
 *            the order-preserving rotations of Algorithm 3 and Algorithm 4 put
 *            the zero rows last in their original order);
 *   L        n x n, unit lower triangular, row k = row perm[k]; columns >= r
 *            are identity columns;
 *   d[k]     D_kk;  e[k] = x when (k, k+1) starts a 2x2 block, else 0.
 *
 * All arithmetic is on canonical residues in [0, p) with 64-bit products and
 * one '%' per operation -- no delayed reduction, no blocking.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Deliberate mistakes, used only by the mutation tests that prove the pins
 * catch them.  0 = the faithful oracle. */
enum {
    MUT_NONE = 0,
    MUT_DROP_CHAR2_TERM = 1,   /* omit + y beta_t beta_u when p = 2          */
    MUT_DELTA_FULL_Y = 2,      /* odd p: delta = y instead of y/2           */
    MUT_LAST_NONZERO = 3,      /* partner = last non-zero instead of first  */
    MUT_SWAP_ALPHA_BETA = 4,   /* write alpha into b's column, beta into a's */
    MUT_NO_DIAG_FIRST = 5,     /* ignore the diagonal: always search j > 0  */
    MUT_UPDATE_SIGN = 6,       /* S_tu += ... instead of -=                 */
};

static uint32_t o_mul(uint32_t a, uint32_t b, uint32_t p)
{
    return (uint32_t)(((uint64_t)a * (uint64_t)b) % p);
}

static uint32_t o_add(uint32_t a, uint32_t b, uint32_t p)
{
    return (uint32_t)(((uint64_t)a + (uint64_t)b) % p);
}

static uint32_t o_sub(uint32_t a, uint32_t b, uint32_t p)
{
    return (uint32_t)(((uint64_t)a + (uint64_t)(p - b)) % p);
}

/* Inverse modulo a prime p by the extended Euclidean algorithm. */
static uint32_t o_inv(uint32_t a, uint32_t p)
{
    int64_t r0 = p, r1 = a % p, s0 = 0, s1 = 1;
    while (r1 != 0) {
        int64_t q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    /* r0 == gcd == 1 for a != 0 and p prime */
    s0 %= (int64_t)p;
    if (s0 < 0) s0 += p;
    return (uint32_t)s0;
}

uint32_t oracle_inv_mod(uint32_t a, uint32_t p) { return o_inv(a, p); }

/*
 * Factor the symmetric matrix whose lower triangle (with diagonal) is stored
 * row-major in A (leading dimension lda).  Entries are reduced mod p.
 *
 * perm[n], d[n], e[n] are always written.  L (n x n, leading dimension ldl)
 * may be NULL.  stop_after < 0 runs to completion; otherwise the elimination
 * stops once that many pivots exist (used only to time a bounded sample), and
 * the outputs are then partial.  *ops_done (may be NULL) receives the sum over
 * the pivots taken of m^2, m being the order of the Schur complement that pivot
 * eliminates from (the per-step term of the operation count of Section 6).
 * Returns the rank r, or -1 when memory runs out.
 */
int64_t oracle_ldlt_rpm(int64_t n, uint32_t p, const uint32_t *A, int64_t lda,
                        int32_t *perm, uint32_t *L, int64_t ldl, uint32_t *d,
                        uint32_t *e, int64_t stop_after, int nthreads,
                        int mutation, double *ops_done)
{
    if (n <= 0) {
        if (ops_done) *ops_done = 0.0;
        return 0;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    size_t nn = (size_t)n * (size_t)n;
    uint32_t *S = (uint32_t *)malloc(nn * sizeof(uint32_t));
    uint32_t *Lw = (uint32_t *)calloc(nn, sizeof(uint32_t)); /* Lw[t][c] by original row t */
    int32_t *rem = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *nonpiv = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *state = (uint8_t *)calloc((size_t)n, 1); /* 0 remaining, 1 pivot, 2 non-pivot */
    if (!S || !Lw || !rem || !nonpiv || !state) {
        free(S); free(Lw); free(rem); free(nonpiv); free(state);
        return -1;
    }

    /* S = A mod p, mirrored from the lower triangle. */
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j) {
            uint32_t v = A[i * lda + j] % p;
            S[i * n + j] = v;
            S[j * n + i] = v;
        }

    int64_t nrem = n;
    for (int64_t i = 0; i < n; ++i) rem[i] = (int32_t)i;
    int64_t r = 0, nz = 0;
    double ops = 0.0;
    uint32_t inv2 = (p == 2) ? 0 : (uint32_t)((p + 1) / 2);

    for (int64_t a = 0; a < n; ++a) {
        if (state[a] != 0) continue;                 /* consumed partner */
        if (stop_after >= 0 && r >= stop_after) break;

        /* drop a from the remaining list */
        int64_t w = 0;
        for (int64_t q = 0; q < nrem; ++q)
            if (rem[q] != a) rem[w++] = rem[q];
        nrem = w;

        uint32_t saa = S[a * n + a];
        int use_diag = (mutation == MUT_NO_DIAG_FIRST) ? 0 : (saa != 0);
        if (use_diag) {
            /* ---- 1x1 pivot ---- */
            uint32_t dd = saa, dinv = o_inv(dd, p);
            ops += (double)(nrem + 1) * (double)(nrem + 1);
            for (int64_t q = 0; q < nrem; ++q) {
                int64_t t = rem[q];
                Lw[t * n + r] = o_mul(S[t * n + a], dinv, p);
            }
            Lw[a * n + r] = 1;
            #pragma omp parallel for schedule(static)
            for (int64_t qt = 0; qt < nrem; ++qt) {
                int64_t t = rem[qt];
                uint32_t coef = o_mul(Lw[t * n + r], dd, p); /* = S_ta */
                for (int64_t qu = 0; qu < nrem; ++qu) {
                    int64_t u = rem[qu];
                    uint32_t upd = o_mul(coef, Lw[u * n + r], p);
                    S[t * n + u] = (mutation == MUT_UPDATE_SIGN)
                                       ? o_add(S[t * n + u], upd, p)
                                       : o_sub(S[t * n + u], upd, p);
                }
            }
            state[a] = 1;
            perm[r] = (int32_t)a;
            d[r] = dd;
            e[r] = 0;
            r += 1;
            continue;
        }

        /* ---- search the Schur row for its first non-zero beyond a ---- */
        int64_t b = -1;
        for (int64_t q = 0; q < nrem; ++q) {
            int64_t u = rem[q];
            if (u > a && S[a * n + u] != 0) {
                b = u;
                if (mutation != MUT_LAST_NONZERO) break;
            }
        }
        if (b < 0) {
            /* ---- zero row: not a pivot ---- */
            state[a] = 2;
            nonpiv[nz++] = (int32_t)a;
            continue;
        }

        /* ---- 2x2 pivot on (a, b) ---- */
        w = 0;
        for (int64_t q = 0; q < nrem; ++q)
            if (rem[q] != b) rem[w++] = rem[q];
        nrem = w;
        ops += (double)(nrem + 2) * (double)(nrem + 2) + (double)(nrem + 1) * (double)(nrem + 1);

        uint32_t x = S[a * n + b], y = S[b * n + b], xinv = o_inv(x, p);
        uint32_t delta, ell;
        if (p == 2) {
            delta = y;
            ell = 0;
        } else {
            delta = (mutation == MUT_DELTA_FULL_Y) ? y : o_mul(y, inv2, p);
            ell = o_mul(delta, xinv, p);
        }
        int64_t ca = r, cb = r + 1; /* L columns of a and b */
        if (mutation == MUT_SWAP_ALPHA_BETA) { ca = r + 1; cb = r; }
        for (int64_t q = 0; q < nrem; ++q) {
            int64_t t = rem[q];
            uint32_t beta = o_mul(S[t * n + a], xinv, p);
            uint32_t alpha = o_mul(o_sub(S[t * n + b], o_mul(beta, delta, p), p), xinv, p);
            Lw[t * n + ca] = alpha;
            Lw[t * n + cb] = beta;
        }
        Lw[a * n + r] = 1;
        Lw[a * n + r + 1] = 0;
        Lw[b * n + r] = ell;
        Lw[b * n + r + 1] = 1;
        int char2 = (p == 2) && (mutation != MUT_DROP_CHAR2_TERM);
        #pragma omp parallel for schedule(static)
        for (int64_t qt = 0; qt < nrem; ++qt) {
            int64_t t = rem[qt];
            uint32_t at = Lw[t * n + ca], bt = Lw[t * n + cb];
            for (int64_t qu = 0; qu < nrem; ++qu) {
                int64_t u = rem[qu];
                uint32_t au = Lw[u * n + ca], bu = Lw[u * n + cb];
                uint32_t upd = o_mul(x, o_add(o_mul(at, bu, p), o_mul(bt, au, p), p), p);
                if (char2) upd = o_add(upd, o_mul(y, o_mul(bt, bu, p), p), p);
                S[t * n + u] = (mutation == MUT_UPDATE_SIGN)
                                   ? o_add(S[t * n + u], upd, p)
                                   : o_sub(S[t * n + u], upd, p);
            }
        }
        state[a] = 1;
        state[b] = 1;
        perm[r] = (int32_t)a;
        perm[r + 1] = (int32_t)b;
        d[r] = 0;
        d[r + 1] = (p == 2) ? y : 0;
        e[r] = x;
        e[r + 1] = 0;
        r += 2;
    }

    /* non-pivot rows last, in ascending original order */
    int64_t k = r;
    for (int64_t q = 0; q < nz; ++q) perm[k++] = nonpiv[q];
    /* rows never reached (only when stopped early) */
    for (int64_t a = 0; a < n && k < n; ++a)
        if (state[a] == 0) perm[k++] = (int32_t)a;
    for (int64_t q = r; q < n; ++q) {
        d[q] = 0;
        e[q] = 0;
    }

    if (L) {
        for (int64_t kk = 0; kk < n; ++kk) {
            int64_t t = perm[kk];
            for (int64_t c = 0; c < n; ++c) {
                uint32_t v;
                if (c < r) v = Lw[t * n + c];
                else v = (c == kk) ? 1u : 0u;
                L[kk * ldl + c] = v;
            }
        }
    }
    if (ops_done) *ops_done = ops;
    free(S); free(Lw); free(rem); free(nonpiv); free(state);
    return r;
}

/* Number of OpenMP threads the oracle would use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
