"""ORACLE -- test infrastructure only (see the package docstring).

Python side of the oracle: the ctypes wrapper around ``ldlt_oracle.c`` and the
plain definitions the tests pin it with.

* ``ldlt_rpm``                -- the factorisation (Algorithm 4 pivoting, Section 5),
                                 computed by the C oracle.
* ``rpm_from_factor``         -- Pi = P Psi P^T (Section 2.1, Definition of the
                                 pivoting matrix; "reveals" = Pi equals R_A).
* ``rank_profile_bruteforce`` -- R_A by Theorem 1: the unique rook placement whose
                                 leading i x j blocks have the ranks of A's.
* ``check_factor``            -- P^T A P == L D L^T exactly mod p (abstract).
* ``freivalds_check``         -- the same identity checked on random vectors, for
                                 sizes where the O(n^3) product is too slow.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldlt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MUTATIONS = {
    "none": 0,
    "drop_char2_term": 1,
    "delta_full_y": 2,
    "last_nonzero": 3,
    "swap_alpha_beta": 4,
    "no_diag_first": 5,
    "update_sign": 6,
}


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_ldlt_rpm.restype = ctypes.c_int64
            lib.oracle_ldlt_rpm.argtypes = [
                ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int64,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                ctypes.POINTER(ctypes.c_double),
            ]
            lib.oracle_inv_mod.restype = ctypes.c_uint32
            lib.oracle_inv_mod.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_max_threads.argtypes = []
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def inv_mod(a: int, p: int) -> int:
    return int(_load().oracle_inv_mod(int(a) % p, p))


def ldlt_rpm(A, p: int, *, want_L: bool = True, stop_after: int = -1,
             nthreads: int = 0, mutation: str = "none") -> dict:
    """Factor the symmetric matrix A (its lower triangle is read) mod p.

    Returns dict(perm, L, d, e, rank, ops) with the conventions of
    ``ldlt_oracle.c``: perm[k] is the original index of row k of P^T A P, L is
    unit lower triangular (n x n, rows in perm order), d the diagonal of D and
    e[k] = x when (k, k+1) is a 2x2 block [[0,x],[x,0]] (odd p) or
    [[0,x],[x,y]] (p = 2).
    """
    A = np.ascontiguousarray(np.asarray(A, dtype=np.uint32))
    n = A.shape[0]
    assert A.shape == (n, n)
    perm = np.zeros(n, dtype=np.int32)
    d = np.zeros(n, dtype=np.uint32)
    e = np.zeros(n, dtype=np.uint32)
    L = np.zeros((n, n), dtype=np.uint32) if want_L else None
    ops = ctypes.c_double(0.0)
    lib = _load()
    r = lib.oracle_ldlt_rpm(
        n, p, A.ctypes.data, n, perm.ctypes.data,
        L.ctypes.data if L is not None else None, n,
        d.ctypes.data, e.ctypes.data, int(stop_after), int(nthreads),
        MUTATIONS[mutation], ctypes.byref(ops))
    if r < 0:
        raise MemoryError("oracle: allocation failed")
    return dict(perm=perm, L=L, d=d, e=e, rank=int(r), ops=float(ops.value))


# ---------------------------------------------------------------------------
# plain definitions used to pin the oracle
# ---------------------------------------------------------------------------

def matmul_mod(X, Y, p: int):
    """Exact (X @ Y) mod p for residue matrices, with int64 numpy products.

    X is split into 16-bit halves so that every partial sum stays below 2^63
    for inner dimension up to 2^16 and p < 2^31.
    """
    X = np.asarray(X, dtype=np.int64) % p
    Y = np.asarray(Y, dtype=np.int64) % p
    k = X.shape[1]
    assert k <= (1 << 16)
    hi = X >> 16
    lo = X & 0xFFFF
    # chunk the inner dimension so 2^16 * 2^31 * chunk < 2^63
    out = np.zeros((X.shape[0], Y.shape[1]), dtype=np.int64)
    step = 1 << 15
    for s in range(0, k, step):
        ph = (hi[:, s:s + step] @ Y[s:s + step]) % p
        pl = (lo[:, s:s + step] @ Y[s:s + step]) % p
        out = (out + ((ph << 16) % p) + pl) % p
    return out


def rank_mod_p(M, p: int) -> int:
    """Rank of M over Z/pZ by plain Gaussian elimination (p prime)."""
    M = np.array(M, dtype=np.int64) % p
    rows, cols = M.shape
    r = 0
    for c in range(cols):
        if r == rows:
            break
        nz = np.nonzero(M[r:, c])[0]
        if nz.size == 0:
            continue
        piv = r + int(nz[0])
        if piv != r:
            M[[r, piv]] = M[[piv, r]]
        inv = pow(int(M[r, c]), p - 2, p)
        M[r] = (M[r] * inv) % p
        below = M[r + 1:, c].copy()
        if below.any():
            M[r + 1:] = (M[r + 1:] - np.outer(below, M[r]) % p) % p
        r += 1
    return r


def rank_profile_bruteforce(A, p: int):
    """R_A from Theorem 1: R_ij = rho(i+1,j+1) - rho(i,j+1) - rho(i+1,j) + rho(i,j),
    rho(i, j) being the rank mod p of the leading i x j block of A.  (A rook
    placement has, in every leading block, as many ones as its rank; the
    inclusion-exclusion of those counts isolates entry (i, j).)"""
    A = np.asarray(A, dtype=np.int64) % p
    m, n = A.shape
    rho = np.zeros((m + 1, n + 1), dtype=np.int64)
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            rho[i, j] = rank_mod_p(A[:i, :j], p)
    R = rho[1:, 1:] - rho[:-1, 1:] - rho[1:, :-1] + rho[:-1, :-1]
    return R.astype(np.int64)


def rpm_from_factor(perm, e, rank: int):
    """rpm_col[i] = j where (P Psi P^T)_ij = 1, else -1.

    Psi is the support of D: a 1 on the diagonal for a 1x1 block, the
    antidiagonal J for a 2x2 block (Section 2.1; for p = 2 the relaxed block
    [[0,c],[c,d]] still has support J, Section 2.2).  With P e_k = e_perm[k],
    Psi_kk = 1 gives R[perm[k], perm[k]] = 1 and a block (k, k+1) gives
    R[perm[k], perm[k+1]] = R[perm[k+1], perm[k]] = 1.
    """
    perm = np.asarray(perm)
    n = perm.shape[0]
    out = np.full(n, -1, dtype=np.int64)
    k = 0
    while k < rank:
        if e[k] != 0:
            a, b = int(perm[k]), int(perm[k + 1])
            out[a] = b
            out[b] = a
            k += 2
        else:
            a = int(perm[k])
            out[a] = a
            k += 1
    return out


def rpm_col_to_matrix(rpm_col):
    n = len(rpm_col)
    R = np.zeros((n, n), dtype=np.int64)
    for i, j in enumerate(rpm_col):
        if j >= 0:
            R[i, j] = 1
    return R


def canonical_perm_from_rpm(R):
    """The pivot order the lexicographic search of Algorithm 4 must produce,
    read off the rank profile matrix alone: rows in ascending order; a row i
    with R_ii = 1 is a 1x1 pivot; a row i with R_ij = 1 for j > i opens the
    pair (i, j); a row matched to an earlier row is skipped (already placed);
    rows with no 1 go last, ascending.  Returns (perm, is_pair_start)."""
    R = np.asarray(R)
    n = R.shape[0]
    perm, starts, zero = [], [], []
    placed = np.zeros(n, dtype=bool)
    for i in range(n):
        if placed[i]:
            continue
        cols = np.nonzero(R[i])[0]
        if cols.size == 0:
            zero.append(i)
            continue
        j = int(cols[0])
        if j == i:
            perm.append(i)
            starts.append(False)
            placed[i] = True
        elif j > i:
            perm += [i, j]
            starts += [True, False]
            placed[i] = placed[j] = True
        else:  # j < i would mean the partner was visited first
            raise AssertionError("inconsistent rank profile matrix")
    return np.array(perm + zero, dtype=np.int64), np.array(starts + [False] * len(zero))


def build_D(d, e, p: int):
    """Dense D from the (d, e) encoding."""
    n = len(d)
    D = np.zeros((n, n), dtype=np.int64)
    for k in range(n):
        D[k, k] = int(d[k]) % p
        if e[k] != 0:
            D[k, k + 1] = int(e[k]) % p
            D[k + 1, k] = int(e[k]) % p
    return D


def symmetrize_lower(A, p: int):
    A = np.asarray(A, dtype=np.int64) % p
    Lo = np.tril(A)
    return Lo + np.tril(A, -1).T


def check_factor(A, perm, L, d, e, p: int) -> bool:
    """P^T A P == L D L^T exactly mod p (A read by its lower triangle)."""
    S = symmetrize_lower(A, p)
    perm = np.asarray(perm, dtype=np.int64)
    PAP = S[np.ix_(perm, perm)]
    D = build_D(d, e, p)
    LD = matmul_mod(np.asarray(L, dtype=np.int64), D, p)
    LDLt = matmul_mod(LD, np.asarray(L, dtype=np.int64).T, p)
    return bool(np.array_equal(PAP % p, LDLt % p))


def freivalds_check(A, perm, L, d, e, p: int, trials: int = 2, seed: int = 12345) -> bool:
    """Randomised check of P^T A P == L D L^T: compare both sides on random
    vectors x, computing L (D (L^T x)) right to left; a wrong factor passes
    one trial with probability <= 1/p."""
    rng = np.random.default_rng(seed)
    S = symmetrize_lower(A, p)
    perm = np.asarray(perm, dtype=np.int64)
    n = S.shape[0]
    Lm = np.asarray(L, dtype=np.int64)
    D = build_D(d, e, p)
    for _ in range(trials):
        x = rng.integers(0, p, size=(n, 1), dtype=np.int64)
        # P^T A P x : y = A (P x) then rows permuted
        px = np.zeros_like(x)
        px[perm] = x
        lhs = matmul_mod(S, px, p)[perm]
        t = matmul_mod(Lm.T, x, p)
        t = matmul_mod(D, t, p)
        rhs = matmul_mod(Lm, t, p)
        if not np.array_equal(lhs, rhs):
            return False
    return True


def strict_char2(perm, L, d, e, p: int = 2, mistake: str = "none"):
    """Section 2.2 (Antitriangular decomposition): in characteristic 2 a
    factorisation with relaxed blocks [[0, c], [c, dd]] (dd != 0) becomes one
    with only 1x1 and antidiagonal 2x2 blocks, at a cost linear in the size of L.

    Restated for P^T A P = L D L^T with perm, L (rows in perm order), d, e as
    returned by ldlt_rpm, for every block (k, k+1) with e[k] = c != 0 and
    d[k+1] = dd != 0:
      1. the block is invariant under [[1, 0], [l, 1]] congruence mod 2, so
         L's in-block entry l is folded into column k (column k -= l column k+1);
      2. [[0, c], [c, dd]] = J [[1, 0], [c/dd, 1]] diag(dd, -c^2/dd) [[1, c/dd], [0, 1]] J,
         so P becomes P J (positions k, k+1 swap), L becomes (J L J) times
         [[1, 0], [c/dd, 1]] on columns (k, k+1), and D's block diag(dd, -c^2/dd).
    Blocks with dd = 0 are already antidiagonal.  For odd p (Algorithm 4 then
    yields antidiagonal blocks only) nothing changes.  Returns new
    (perm, L, d, e).  `mistake` plants a known error for the pin tests.
    """
    perm = np.array(perm, dtype=np.int64).copy()
    L = np.array(L, dtype=np.int64).copy() % p
    d = np.array(d, dtype=np.int64).copy() % p
    e = np.array(e, dtype=np.int64).copy() % p
    if p != 2:
        return perm, L, d, e
    n = len(perm)
    blocks = [k for k in range(n - 1) if e[k] != 0 and d[k + 1] != 0]
    for k in blocks:                                   # step 1
        ell = L[k + 1, k]
        L[:, k] = (L[:, k] - ell * L[:, k + 1]) % p
    for k in blocks:                                   # step 2: J L J and P J
        if mistake != "no_row_swap":
            L[[k, k + 1], :] = L[[k + 1, k], :]
        L[:, [k, k + 1]] = L[:, [k + 1, k]]
        if mistake != "no_perm_swap":
            perm[[k, k + 1]] = perm[[k + 1, k]]
    for k in blocks:                                   # step 2: times [[1, 0], [c/dd, 1]]
        c, dd = int(e[k]), int(d[k + 1])
        ratio = c * inv_mod(dd, p) % p
        if mistake != "no_column_op":
            L[:, k] = (L[:, k] + ratio * L[:, k + 1]) % p
        d[k] = dd
        d[k + 1] = (-c * c * inv_mod(dd, p)) % p
        e[k] = 0
    return perm, L, d, e


def solve_factor(perm, L, d, e, rank: int, B, p: int):
    """A X = B from P^T A P = L D L^T (abstract; the motivation of Section 1:
    solving symmetric systems with the factorisation), one step at a time:
      Y = P^T B;  L Z = Y (unit lower triangular, forward);  D W = Z (1x1
      pivots d_k; 2x2 blocks [[0, x], [x, y]]: w1 = z0 / x, w0 = (z1 - y w1) / x;
      rows k >= rank: the system is consistent only if z_k = 0, and w_k = 0);
      L^T V = W (backward);  X = P V.
    Returns (X, consistent).  X is the solution with zero components on the
    non-pivot rows (unique when rank = n)."""
    perm = np.asarray(perm, dtype=np.int64)
    Lm = np.asarray(L, dtype=np.int64) % p
    d = np.asarray(d, dtype=np.int64) % p
    e = np.asarray(e, dtype=np.int64) % p
    B = np.asarray(B, dtype=np.int64) % p
    if B.ndim == 1:
        B = B[:, None]
    n = len(perm)
    Y = B[perm].copy()
    Z = Y.copy()
    for k in range(n):                      # forward, unit diagonal
        if k:
            Z[k] = (Y[k] - matmul_mod(Lm[k:k + 1, :k], Z[:k], p)[0]) % p
    W = np.zeros_like(Z)
    consistent = True
    k = 0
    while k < n:
        if k >= rank:
            if np.any(Z[k] != 0):
                consistent = False
            W[k] = 0
            k += 1
        elif e[k] != 0:
            x, y = int(e[k]), int(d[k + 1])
            ix = inv_mod(x, p)
            W[k + 1] = (Z[k] * ix) % p
            W[k] = ((Z[k + 1] - (y * W[k + 1]) % p) % p * ix) % p
            k += 2
        else:
            W[k] = (Z[k] * inv_mod(int(d[k]), p)) % p
            k += 1
    V = W.copy()
    for k in range(n - 1, -1, -1):          # backward with L^T
        if k < n - 1:
            V[k] = (W[k] - matmul_mod(Lm[k + 1:, k][None, :], V[k + 1:], p)[0]) % p
    X = np.zeros_like(V)
    X[perm] = V
    return X, consistent
