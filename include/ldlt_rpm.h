/*
 * ldlt_rpm.h -- C ABI of the GB300 (sm_103a) symmetric indefinite factorisation
 * over Z/pZ that reveals the rank profile matrix.
 *
 * Method: Dumas & Pernet, "Symmetric indefinite triangular factorization
 * revealing the rank profile matrix" (arXiv 1802.10453).  The factorisation is
 * P^T A P = L D L^T (abstract; A = P L D L^T P^T in Algorithms 2-4) with P a
 * permutation, L unit lower triangular and D block diagonal with 1x1 blocks
 * and 2x2 blocks [[0,x],[x,0]] (odd p) or [[0,x],[x,y]] (p = 2, the relaxed
 * lower antitriangular blocks of Section 2.2).  Pivots follow the
 * lexicographic search of Algorithm 4 (Section 5): for the next row, the
 * diagonal of its Schur complement row if non-zero, else the first non-zero
 * to its right, else the row is not a pivot.  The rank profile matrix is the
 * pivoting matrix P Psi P^T (Section 2.1, Definitions 1 and 2), Psi being the
 * support of D.
 *
 * All matrix and vector pointers are DEVICE pointers owned by the caller.
 * Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = the
 * legacy default stream).  Functions return 0 (LDLT_OK) or a negative
 * LDLT_ERR_* code for errors the host can detect; no C++ exception crosses
 * this boundary.  Errors found on the device (a bounded wait that ran out) are
 * written to the caller's device status word.  Outputs are undefined when
 * either is non-zero.
 */
#ifndef LDLT_RPM_H
#define LDLT_RPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define LDLT_OK              0
#define LDLT_ERR_ARG        -1  /* n < 0, lda < n, a NULL pointer, unknown path   */
#define LDLT_ERR_NOT_PRIME  -2  /* p < 2 or p composite                           */
#define LDLT_ERR_P_RANGE    -3  /* p >= 2^31, or the FP64 path with p too large    */
#define LDLT_ERR_WORKSPACE  -4  /* ws NULL or smaller than the queried size        */
#define LDLT_ERR_CUDA       -5  /* a CUDA runtime call failed (launch, copy, ...)  */
#define LDLT_ERR_TIMEOUT    -6  /* device only: a bounded spin-wait gave up        */
#define LDLT_ERR_NO_DEVICE  -7  /* no sm_103 device visible                         */
#define LDLT_ERR_TOO_LARGE  -8  /* n above LDLT_NOALLOC_MAX_N (no-allocation entry) */
#define LDLT_ERR_INCONSISTENT -9 /* device only (ldlt_rpm_solve): B not in A's column space */
#define LDLT_ERR_INTERNAL  -10  /* device only: a panel retired no row (not expected; the
                                     factorisation stops instead of looping) */

/* ---- arithmetic paths for the level-3 updates (SYRDK, Algorithm 2) ------ */
/* FP64 form: residues carried in doubles, products accumulated with one
 * reduction per block of k terms, k*((p-1)/2)^2 + 1.5p < 2^53 (p < 2^26.5). */
#define LDLT_PATH_FP64      0
/* Tensor form: residues split into signed 8-bit limbs held exactly in bf16,
 * tcgen05.mma kind::f16 with FP32 accumulation (exact below 2^24), limbs
 * recombined and reduced mod p once per output.  Any prime p < 2^31. */
#define LDLT_PATH_TC        1

/*
 * ldlt_rpm_workspace_bytes -- size of the device workspace ldlt_rpm_factor
 * needs for order n, prime p and the given path.  Pure host computation.
 * Returns LDLT_OK and *bytes, or LDLT_ERR_ARG / LDLT_ERR_NOT_PRIME /
 * LDLT_ERR_P_RANGE.
 */
int ldlt_rpm_workspace_bytes(int64_t n, uint32_t p, int path, size_t *bytes);

/*
 * ldlt_rpm_factor -- factor P^T A P = L D L^T mod p in place (the problem of
 * the abstract; pivot order of Algorithm 4, Section 5; level-3 updates of
 * Algorithm 2, Section 4).
 *
 *   n        order of A (n >= 0).
 *   p        prime modulus, 2 <= p < 2^31.
 *   A        n x n row-major uint32 with leading dimension lda (elements).
 *            Input: the lower triangle with the diagonal is read; entries are
 *            reduced mod p.  The upper triangle is ignored.
 *            Output: strictly below the diagonal, L (row k of L is row k of
 *            P^T A P; unit diagonal implicit; columns k >= rank are identity
 *            columns); on the diagonal, D_kk.  The upper triangle is left
 *            unspecified.
 *   perm     int32[n]: perm[k] = original index of row/column k of P^T A P
 *            (P e_k = e_perm[k]).  Pivots come in the order found, a before b
 *            for a 2x2 pivot on rows a < b, then the non-pivot rows in
 *            ascending order.
 *   e        uint32[n]: e[k] = x when rows (k, k+1) form a 2x2 block, else 0.
 *   rank     int64[1]: the rank r.
 *   status   int32[1]: 0, or LDLT_ERR_TIMEOUT if a device wait gave up.
 *   path     LDLT_PATH_FP64 or LDLT_PATH_TC.
 *   ws       device workspace of at least ldlt_rpm_workspace_bytes() bytes,
 *            256-byte aligned; owned by the caller, not retained after return.
 *   stream   cudaStream_t as void*.
 *
 * The call only enqueues work on `stream`: nothing is read back and the host
 * does not wait; results (A, perm, e, rank, status) are ready when the stream
 * is.  The panel loop runs on the device as one CUDA graph (a while node
 * whose condition the last kernel of each iteration sets); the graph is built
 * and instantiated on the first call with a given set of arguments (n, p,
 * path, lda, every pointer, the wait budget, the speculation depth) and
 * launched again, unchanged, by later calls with the same set (the library
 * keeps the four most recently used).  A kept graph refers to the caller's
 * buffers only by address.  With profiling on (ldlt_rpm_profile_enable) the
 * same kernels run from a host loop that synchronises `stream` once per
 * panel to time the phases.
 */
int ldlt_rpm_factor(int64_t n, uint32_t p, uint32_t *A, int64_t lda,
                    int32_t *perm, uint32_t *e, int64_t *rank, int32_t *status,
                    int path, void *ws, size_t ws_bytes, void *stream);

/*
 * rpm_from_factor -- the rank profile matrix R_A = P Psi P^T (Section 2.1,
 * Definition 1; Psi = support of D, for p = 2 the relaxed block's support is
 * still the antidiagonal J, Section 2.2).
 *
 *   n, perm, e, rank   as returned by ldlt_rpm_factor (device pointers;
 *                      rank is read on the device).
 *   rpm_col            int32[n] output: rpm_col[i] = j if (R_A)_{ij} = 1,
 *                      else -1.  R_A is a symmetric rook placement (Lemma 1).
 * Returns LDLT_OK, LDLT_ERR_ARG or LDLT_ERR_CUDA.
 */
int rpm_from_factor(int64_t n, const int32_t *perm, const uint32_t *e,
                    const int64_t *rank, int32_t *rpm_col, void *stream);

/*
 * ldlt_rpm_solve -- A X = B with the factorisation of A (Section 1: a
 * symmetric triangular factorisation is the kernel for solving symmetric
 * systems).  From P^T A P = L D L^T:  Z = P^T B, L Z' = Z, D W = Z',
 * L^T V = W, X = P V.  On the rows k >= rank the system is consistent only if
 * Z'_k = 0; X is then the solution whose non-pivot components (in pivot
 * order) are 0, the unique one when rank = n.
 *
 *   n, p, A, lda, perm, e, rank   the outputs of ldlt_rpm_factor for A (A as
 *                                 overwritten by it; rank read on the device).
 *   B        n x nrhs row-major uint32 (device), leading dimension ldb >= nrhs;
 *            entries are reduced mod p.  Not modified.
 *   X        n x nrhs row-major uint32 output (device), ldx >= nrhs; may not
 *            alias B.
 *   status   int32[1] (device): 0, or LDLT_ERR_INCONSISTENT when B has a
 *            column outside A's column space (X is then unspecified).
 *   ws       device workspace of at least 4 * n * nrhs bytes.
 *   stream   cudaStream_t as void*; about 4 n / 64 kernels are enqueued (one
 *            diagonal-block solve and one update per block of 64 rows, both
 *            directions); nothing is read back.
 * Returns LDLT_OK, LDLT_ERR_ARG, LDLT_ERR_NOT_PRIME, LDLT_ERR_P_RANGE,
 * LDLT_ERR_WORKSPACE or LDLT_ERR_CUDA.
 */
int ldlt_rpm_solve(int64_t n, uint32_t p, const uint32_t *A, int64_t lda,
                   const int32_t *perm, const uint32_t *e, const int64_t *rank,
                   const uint32_t *B, int64_t ldb, int64_t nrhs,
                   uint32_t *X, int64_t ldx, int32_t *status,
                   void *ws, size_t ws_bytes, void *stream);

/*
 * ldlt_rpm_factor_given -- the given-P mode: the L and D of P^T A P = L D L^T
 * for a pivot order and block structure supplied by the caller, e.g. those of
 * Algorithm 2/3 (Section 4), whose order can differ from Algorithm 4's.  For
 * odd p they are unique once P and the blocks are fixed (a 2x2 block
 * [[0, x], [x, y]] of the Schur complement has in-block entry y/(2x) and
 * D block [[0, x], [x, 0]]); for p = 2 the block keeps [[0, x], [x, y]] and
 * in-block entry 0 (the conventions of ldlt_rpm_factor).
 *
 *   n, p, A, lda, path, ws, stream   as for ldlt_rpm_factor; A's lower
 *            triangle is read in the original order and overwritten with L
 *            and D in the supplied order (layout of ldlt_rpm_factor).
 *   perm     int32[n], in: perm[k] = original index of position k (a
 *            permutation of 0..n-1); out: unchanged.
 *   e        uint32[n], in: e[k] != 0 marks a 2x2 block (k, k+1); out: x of
 *            each block, 0 elsewhere.
 *   rank     int64[1], in: the number of pivot positions (blocks count two);
 *            out: the same when the structure fits.
 *   status   int32[1]: 0; LDLT_ERR_ARG if perm is not a permutation;
 *            LDLT_ERR_INCONSISTENT if the structure does not fit A (a zero
 *            1x1 pivot, a 2x2 start with a non-zero diagonal or a zero x, or a
 *            non-zero Schur complement after the rank); LDLT_ERR_TIMEOUT as
 *            for ldlt_rpm_factor.  Outputs are undefined when non-zero.
 *   ws_bytes at least ldlt_rpm_given_workspace_bytes(n, p, path).
 * Runs ldlt_rpm_factor's path on P^T A P gathered in its ingest pass:
 * Algorithm 4's search takes the identity order there exactly when the
 * structure fits, and the result is checked against the supplied one.
 * Returns as ldlt_rpm_factor.
 */
int ldlt_rpm_given_workspace_bytes(int64_t n, uint32_t p, int path, size_t *bytes);
int ldlt_rpm_factor_given(int64_t n, uint32_t p, uint32_t *A, int64_t lda,
                          int32_t *perm, uint32_t *e, int64_t *rank, int32_t *status,
                          int path, void *ws, size_t ws_bytes, void *stream);

/*
 * ldlt_rpm_trss -- Algorithm 1 (TRSS) of Section 4, Problem 1: the upper
 * triangular X with X^T U + U^T X = C over Z/pZ, the routine Algorithm 3
 * uses to eliminate the leading block of Q C Q^T with the pivots of B.
 *
 *   n        order (>= 0).
 *   p        prime, 2 <= p < 2^31.  For p = 2 a solution exists only when the
 *            diagonal met at each step is zero (the diagonal of X^T U + U^T X
 *            is zero in characteristic 2); x_ii = 0 is taken there.
 *   U, ldu   n x n upper triangular with a non-zero diagonal, row-major; only
 *            the upper triangle (i <= j) is read; entries reduced mod p.
 *   C, ldc   n x n symmetric, row-major; its upper triangle (i <= j) is read
 *            and overwritten by X (in place); the strict lower triangle is
 *            not touched.
 *   status   int32[1]: 0; LDLT_ERR_ARG if U has a zero diagonal entry;
 *            LDLT_ERR_INCONSISTENT if p = 2 and no solution exists.  X is
 *            undefined then.
 *   stream   cudaStream_t as void*; three launches per 32-row block are
 *            enqueued, nothing is read back.
 * Returns LDLT_OK, LDLT_ERR_ARG (n < 0, ld < n, NULL pointer),
 * LDLT_ERR_NOT_PRIME, LDLT_ERR_P_RANGE or LDLT_ERR_CUDA.
 */
int ldlt_rpm_trss(int64_t n, uint32_t p, const uint32_t *U, int64_t ldu,
                  uint32_t *C, int64_t ldc, int32_t *status, void *stream);

/*
 * ldlt_rpm_trss_ws -- ldlt_rpm_trss with the trailing update of every block
 * step (Algorithm 1's C3 - (X2^T U2 + U2^T X2), a SYR2K) on tcgen05 tensor
 * cores: the exact bf16-limb product of ldlt_rpm_factor's level-3 update,
 * with G = [X^T | U^T] and G D = [U^T | X^T] (K = 2 x 32 per step), written
 * to C's upper triangle in place.  Trailing orders below 256 keep the
 * CUDA-core update.  Same arguments, outputs and errors as ldlt_rpm_trss
 * (bit-identical results), plus
 *   ws, ws_bytes  device workspace of at least ldlt_rpm_trss_workspace_bytes
 *                 bytes, 256-byte aligned, owned by the caller (limb
 *                 operands and the update's size record);
 *   status        also LDLT_ERR_TIMEOUT if the update kernel's bounded wait
 *                 gave up.
 * Returns what ldlt_rpm_trss returns, LDLT_ERR_WORKSPACE, or
 * LDLT_ERR_NO_DEVICE if the device is not sm_103.  Five launches per 32-row
 * block are enqueued; nothing is read back.
 */
int ldlt_rpm_trss_workspace_bytes(int64_t n, uint32_t p, size_t *bytes);
int ldlt_rpm_trss_ws(int64_t n, uint32_t p, const uint32_t *U, int64_t ldu,
                     uint32_t *C, int64_t ldc, int32_t *status, void *ws, size_t ws_bytes,
                     void *stream);

/*
 * ldlt_rpm_strict -- the strict form of a characteristic-2 factorisation
 * (Section 2.2, "Antitriangular decomposition"), in place on the outputs of
 * ldlt_rpm_factor / ldlt_rpm_factor_batched for the same A.
 *
 * Over F_2 Algorithm 4 may return relaxed blocks [[0, c], [c, d]] with d != 0
 * (Section 2.2; the only factorisation shape that exists in characteristic
 * 2).  Each such block is replaced by two 1x1 pivots: its two positions swap
 * in perm, rows and columns k, k+1 of L are swapped and column k becomes
 * column k + column k+1 below the block, D's block becomes diag(1, 1) and
 * e[k] becomes 0.  Afterwards P^T A P = L D L^T still holds with only 1x1
 * pivots and antidiagonal blocks [[0, c], [c, 0]] in D, but perm and D no
 * longer reveal the rank profile matrix: call rpm_from_factor before this.
 *
 *   n, p, A, lda, perm, e   as passed to / returned by ldlt_rpm_factor (p the
 *                           same prime).  For odd p nothing changes: the
 *                           blocks of Algorithm 4 are antidiagonal already.
 *   stream                  cudaStream_t as void*; three launches are
 *                           enqueued, nothing is read back.
 * Returns LDLT_OK, LDLT_ERR_ARG, LDLT_ERR_NOT_PRIME, LDLT_ERR_P_RANGE or
 * LDLT_ERR_CUDA.
 */
int ldlt_rpm_strict(int64_t n, uint32_t p, uint32_t *A, int64_t lda,
                    int32_t *perm, uint32_t *e, void *stream);

/*
 * ldlt_rpm_factor_batched -- factor `count` independent matrices, each as
 * ldlt_rpm_factor does (same pivot order, same outputs bit for bit), in one
 * persistent launch: the batched use of the method that Section 6 discusses
 * (many problems whose order is below the recursion threshold).  Every CTA
 * factors whole matrices taken from a queue in order of decreasing n; a
 * matrix never leaves its SM.
 *
 *   count    number of matrices (0 <= count <= INT_MAX).
 *   n        int64[count] (device): orders, 0 <= n[i] <= LDLT_BATCH_MAX_N.
 *   p        prime modulus shared by all matrices, as for ldlt_rpm_factor.
 *   A        uint32*[count] (device array of device pointers): matrix i,
 *            row-major with leading dimension lda[i] >= n[i]; input and output
 *            as for ldlt_rpm_factor.
 *   lda      int64[count] (device).
 *   perm     int32*[count], e uint32*[count] (device arrays of device
 *            pointers): outputs as for ldlt_rpm_factor, n[i] entries each.
 *   rank     int64[count] (device): ranks.
 *   status   int32[count] (device): 0, or LDLT_ERR_ARG for a matrix whose
 *            n, lda or pointers are invalid (that matrix is left untouched;
 *            the others are factored).
 *   path     LDLT_PATH_FP64 or LDLT_PATH_TC, range-checked as for
 *            ldlt_rpm_factor (an unknown value, or LDLT_PATH_FP64 with p
 *            beyond the FP64 range, is an error) but it does not select the
 *            arithmetic: the batched update's form follows from p alone,
 *            bf16 limbs on the tensor cores (mma.sync) for p < 2^16 and exact
 *            64-bit products on the CUDA cores above.  Both give the same
 *            bits; matrices of order <= 512 are bound by the pivot chain.
 *   ws       device workspace, 256-byte aligned: at least the header plus one
 *            CTA's scratch (1 MiB); ldlt_rpm_batched_workspace_bytes gives the
 *            size that lets every resident CTA run.  A smaller workspace runs
 *            fewer CTAs.  While a matrix is factored, the lower triangle of its
 *            A holds its Schur complement; the upper triangle is not touched.
 *   stream   cudaStream_t as void*.
 *
 * Enqueues three operations on `stream` (a memset and two kernels) and
 * returns without synchronising; nothing is read back to the host.  Returns
 * LDLT_OK, LDLT_ERR_ARG, LDLT_ERR_NOT_PRIME, LDLT_ERR_P_RANGE,
 * LDLT_ERR_WORKSPACE, LDLT_ERR_CUDA or LDLT_ERR_NO_DEVICE.
 */
#define LDLT_BATCH_MAX_N    512
int ldlt_rpm_factor_batched(int64_t count, const int64_t *n, uint32_t p,
                            uint32_t *const *A, const int64_t *lda,
                            int32_t *const *perm, uint32_t *const *e,
                            int64_t *rank, int32_t *status, int path,
                            void *ws, size_t ws_bytes, void *stream);

/*
 * ldlt_rpm_batched_workspace_bytes -- workspace of ldlt_rpm_factor_batched
 * for `count` matrices: a header (queue counter, queue order) and 1 MiB of
 * scratch for each CTA that can run (at most min(count, 640)).  Pure host
 * computation.  Returns LDLT_OK, LDLT_ERR_ARG, LDLT_ERR_NOT_PRIME or
 * LDLT_ERR_P_RANGE.
 */
int ldlt_rpm_batched_workspace_bytes(int64_t count, uint32_t p, int path, size_t *bytes);

/*
 * ldlt_rpm_batched_set_schedule -- tile and cutoff choices of the batched
 * schedule (process-wide; picked by the package's autotuner): kb = 16, 32 or
 * 64 is the largest number of pivots per panel the kernel is built for (it
 * fixes shared memory and so the CTAs per SM); matrices with n < n_cut use
 * panels of kb_small (4 <= kb_small <= kb) pivots instead.  Results do not
 * depend on these choices.  Default (32, 0, 32).  Returns LDLT_OK or
 * LDLT_ERR_ARG.
 */
int ldlt_rpm_batched_set_schedule(int kb, int n_cut, int kb_small);

/*
 * ldlt_rpm_factor_noalloc -- ldlt_rpm_factor for callers that must not
 * allocate device memory at call time.  The paper has no counterpart: it is a
 * packaging of the same factorisation, not a step of the method.
 *
 * Some callers cannot hand the library a workspace: a plain C program that
 * has given all of its device memory to its own pool, or a latency-critical
 * loop in which a cudaMalloc (which may synchronise the whole device) is not
 * acceptable.  This entry point takes the arguments of ldlt_rpm_factor minus
 * ws / ws_bytes and runs the same kernels with their scratch in one
 * file-scope device array of LDLT_NOALLOC_BYTES bytes that is part of the
 * library.  It calls no cudaMalloc / cudaFree and no allocating library
 * routine.
 *
 *   n        0 <= n <= LDLT_NOALLOC_MAX_N; a larger n returns
 *            LDLT_ERR_TOO_LARGE before any device work.
 *   others   exactly as for ldlt_rpm_factor (same outputs, bit for bit).
 *
 * Set-up: every call looks up the array's device address on the current
 * device (cudaGetSymbolAddress, which allocates nothing once the module is
 * loaded), so the address stays right after cudaDeviceReset or under another
 * context.  CUDA reserves the array's memory when it loads the module that
 * holds it; with CUDA's default lazy module loading that happens at the first
 * call on a device, not when the library is opened.  Make that first call
 * before any stream capture begins.  A failed lookup returns LDLT_ERR_CUDA
 * and leaves an error the caller had pending untouched.  Like
 * ldlt_rpm_factor, the call only enqueues work, as one CUDA graph: the first
 * call with a given set of arguments builds and instantiates it (the driver
 * keeps what an instantiated graph needs, as it does for a loaded module),
 * and later calls with the same set launch it again and create nothing.
 *
 * Every call on a device uses the same array.  The factorisation clears, on
 * the stream, every part of its scratch that must start at zero, so one call
 * leaves nothing that a later call depends on; but calls that overlap in time
 * on one device (two streams, or two host threads) race on the array and give
 * undefined results.  Serialise them.
 *
 * Returns what ldlt_rpm_factor returns, or LDLT_ERR_TOO_LARGE.
 */
#define LDLT_NOALLOC_MAX_N  1024
#define LDLT_NOALLOC_BYTES  ((size_t)48 << 20)
int ldlt_rpm_factor_noalloc(int64_t n, uint32_t p, uint32_t *A, int64_t lda,
                            int32_t *perm, uint32_t *e, int64_t *rank,
                            int32_t *status, int path, void *stream);

/*
 * ldlt_rpm_version -- library version as major*10000 + minor*100 + patch.
 */
int ldlt_rpm_version(void);

/*
 * ldlt_rpm_set_wait_budget_ns -- upper bound, in nanoseconds, on every
 * spin-wait inside the factorisation kernels (default 2e9).  When a wait runs
 * out the kernel writes LDLT_ERR_TIMEOUT to *status and returns.  Used by the
 * failure-detection tests; 0 restores the default.
 */
void ldlt_rpm_set_wait_budget_ns(int64_t ns);

/*
 * ldlt_rpm_test_drop -- failure-detection test hook (no counterpart in the
 * paper).  Makes the factorisation drop one kind of internal message so that
 * a bounded device wait is certain to run out, which lets a test check that
 * the timeout is reported and that the next call is correct.  Nothing faults
 * or hangs: the wait gives up after the budget of
 * ldlt_rpm_set_wait_budget_ns, the kernel writes LDLT_ERR_TIMEOUT to *status,
 * its other CTAs and warps see the abort flag, drain their own in-flight
 * copies and return, and later kernels of the same call return at once.
 *   LDLT_TEST_DROP_SCAN_ANSWERS   the pivot chain's helper CTAs never answer
 *                                 a far scan (tensor or FP64 form);
 *   LDLT_TEST_DROP_UPDATE_COPIES  the tensor-core SYRDK's copy producer stops
 *                                 after one pipeline stage (LDLT_PATH_TC).
 *   0                             normal operation (the default).
 * Process-wide, not thread-safe.  Returns LDLT_OK or LDLT_ERR_ARG.
 */
#define LDLT_TEST_DROP_SCAN_ANSWERS   1
#define LDLT_TEST_DROP_UPDATE_COPIES  2
int ldlt_rpm_test_drop(int which);

/*
 * ldlt_rpm_set_speculation -- how many far scans the pivot chain may have in
 * flight while it continues past rows whose window part is zero (1..16,
 * default LDLT_SPECULATION_DEFAULT).  A scan that finds a partner rolls the
 * panel back to its row, so the depth trades waiting against discarded work,
 * and every speculative row is also work for the helper CTAs that answer the
 * scans: deeper speculation slows the answers.  Measured on GB300 (n = 16384
 * planted, p = 2^26 - 5): 83 ms at depth 3, 77.8 at 5, 81.9 at 16; n = 32768
 * with only 2x2 pivots, p = 2^31 - 1: 348, 337, 483 ms.  Results do not depend
 * on it.  No counterpart in the paper (a scheduling parameter of this GPU
 * organisation).  Returns LDLT_OK or LDLT_ERR_ARG.
 */
#define LDLT_SPECULATION_DEFAULT 5
int ldlt_rpm_set_speculation(int depth);

/*
 * Profiling counters (no counterpart in the paper; they feed the roofline
 * report).  When enabled, ldlt_rpm_factor records CUDA events around its
 * phases on the caller's stream and accumulates, across calls:
 *   out[0] ms in the pivot-chain kernels (panel + bookkeeping)
 *   out[1] ms in operand preparation (L store, limb split)
 *   out[2] ms in the level-3 update kernel (SYRDK, either form)
 *   out[3] algorithmic multiply-adds of the level-3 updates:
 *          sum over launches of (m'(m'+1)/2) * k (lower triangle, k pivots)
 *   out[4] number of level-3 update launches
 *   out[5] number of kernels this library launched
 *   out[6] number of panels
 *   out[7] far scans issued by the pivot chain
 *   out[8..15] SM clock cycles the pivot chain's leader spent per phase:
 *          candidate column, rollback, 1x1 store, search, scan request,
 *          (unused), zero row, 2x2 pivot
 *   out[16..31] pivot-chain diagnostics: leader row iterations, waits for
 *          a full set of pending scans and their cycles, cycles waiting for
 *          event-ring space, rollbacks, idle and busy cycles and events of
 *          helper CTA 1, publisher batches, events published, (reserved)
 * ldlt_rpm_profile_read returns LDLT_OK, or LDLT_ERR_ARG for a NULL pointer.
 * The counters are process-wide and not thread-safe.
 */
void ldlt_rpm_profile_enable(int on);
void ldlt_rpm_profile_reset(void);
int ldlt_rpm_profile_read(double out[32]);

/*
 * ldlt_rpm_profile_read_hbm -- the HBM-streaming kernels, from the same
 * profiled calls (CUDA events around each launch; the algorithmic bytes are
 * counted on the host from the sizes each launch was given):
 *   out[0..3]   ms in ingest, finalize, L scatter, operand split
 *   out[4..7]   their launches
 *   out[8..11]  their algorithmic bytes: ingest 8 n(n+1)/2 (lower triangle of
 *               A read, of S written); finalize 8 n(n+1)/2 (L rows read, an
 *               upper bound since non-pivot rows read fewer columns, A's lower
 *               triangle written); L scatter 8 np m per panel (np columns of
 *               m rows read, and written by row); split 4 np m' (the columns
 *               of the m' remaining rows) plus the operands written: tensor
 *               form 2 L_A kpad R (1 + L_B) with R = m' rounded up to 128,
 *               FP64 form 16 kpad ldS
 *   out[12]     algorithmic bytes of the level-3 updates: per launch the old
 *               lower triangle of the m' remaining rows read and the new one
 *               written, 8 m'(m'+1)/2, plus the operands once (as above)
 *   out[13]     level-3 update launches
 *   out[14]     the part of out[12] that falls on the first three update
 *               launches of each call (the largest: what a traffic capture
 *               of three launches measures)
 *   out[15]     reserved (0)
 * Returns LDLT_OK, or LDLT_ERR_ARG for a NULL pointer.
 */
int ldlt_rpm_profile_read_hbm(double out[16]);

#ifdef __cplusplus
}
#endif

#endif /* LDLT_RPM_H */
