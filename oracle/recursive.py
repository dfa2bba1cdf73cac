"""ORACLE -- test infrastructure only (imported by tests/ alone; the product path
never calls it).

The block recursive algorithm of Section 4, written plainly over exact Python
integers (numpy object arrays, every entry reduced mod p), for small sizes:

* ``trss``             -- Algorithm 1 (TRSS, Problem 1): X upper triangular with
                          X^T U + U^T X = C.
* ``plduq``            -- a PLDUQ decomposition of a rectangular B that reveals
                          its rank profile matrix.  Section 4 uses one but does
                          not define it; this one takes the rows in order and
                          pivots each on the first non-zero of its Schur row
                          (reading G1).
* ``ldlt_alg2``        -- Algorithm 2 (recursive symmetric indefinite
                          elimination), with ``ldlt_alg3`` -- Algorithm 3 (zero
                          leading block, off-diagonal pivoting), including the
                          characteristic-2 branches (Delta, DADD).
* ``factor_given_p``   -- the "given-P" mode: the unique L and D of
                          P^T A P = L D L^T for a supplied pivot order and block
                          structure (1x1 pivots and 2x2 blocks whose leading
                          entry is zero), by plain block elimination.

Readings (the paper is silent or garbled here):
* m = floor(N / 2) for the split of Algorithm 2.
* Algorithm 3's L lists the lower-left blocks [G2 V1^T ; M1 0] without the
  permutations that act on them: their columns follow the interleaving P_i of
  the leading 2r columns and the rows of [G2 V1^T] follow P3, as the identity
  requires (checked by the tests).
* Characteristic 2: the leading 2x2 blocks are [[0, d_i], [d_i, Delta_ii]];
  TRSS on a zero diagonal takes x_ii = 0 (any value solves 2 x u = 0 there).
* Non-pivot rows are returned in ascending original order.  The final block
  rotation of Algorithm 3 alone would put Bm's non-pivot rows after Z's zero
  rows; the next level takes those rows as the rows of its off-diagonal block
  in that order, and the rank profile is revealed only when they keep their
  original precedence (the requirement the paper states for P_c).
* In the given-P mode a 2x2 block takes L's in-block entry y / (2x) for odd p
  and 0 for p = 2 (the Algorithm 4 conventions).
"""
from __future__ import annotations

import numpy as np


def _z(r, c):
    return np.zeros((r, c), dtype=object)


def _mod(X, p):
    X = np.array(X, dtype=object)
    return np.vectorize(lambda v: int(v) % p, otypes=[object])(X) if X.size else X


def _inv(a, p):
    a = int(a) % p
    if a == 0:
        raise ZeroDivisionError("inverse of 0 mod p")
    return pow(a, p - 2, p)


def _mm(X, Y, p):
    if X.shape[1] == 0:
        return _z(X.shape[0], Y.shape[1])
    return _mod(X.dot(Y), p)


def _lower_solve(Lm, B, p):
    """X with Lm X = B, Lm lower triangular with a non-zero diagonal."""
    n = Lm.shape[0]
    X = _z(n, B.shape[1])
    for i in range(n):
        s = B[i].copy()
        for k in range(i):
            s = s - Lm[i, k] * X[k]
        X[i] = _mod(s * _inv(Lm[i, i], p), p)
    return X


def _upperT_solve(U, B, p):
    """X with U^T X = B, U upper triangular with a non-zero diagonal."""
    return _lower_solve(_mod(U.T, p), B, p)


# ---------------------------------------------------------------------------
# Algorithm 1: TRSS
# ---------------------------------------------------------------------------

def trss(U, C, p: int, mistake: str = "none"):
    """Upper triangular X with X^T U + U^T X = C (U full-rank upper
    triangular, C symmetric).  Algorithm 1: split in halves; X1 from the
    leading halves, D2 = C2 - X1^T U2 (TRMM), X2 = U1^{-T} D2 (TRSM),
    D3 = C3 - (X2^T U2 + U2^T X2) (SYR2K), X3 from the trailing halves.  The
    base case halves: x = c / (2 u).  For p = 2 the diagonal of C must be zero
    and x_ii = 0 is taken."""
    U = _mod(U, p)
    C = _mod(C, p)
    n = U.shape[0]
    if n == 0:
        return _z(0, 0)
    if n == 1:
        c, u = int(C[0, 0]), int(U[0, 0])
        if p == 2:
            if c != 0:
                raise ValueError("TRSS in characteristic 2 needs a zero diagonal")
            return _z(1, 1)
        half = 1 if mistake == "no_halving" else _inv(2, p)
        return np.array([[c * half * _inv(u, p) % p]], dtype=object)
    h = n // 2
    U1, U2, U3 = U[:h, :h], U[:h, h:], U[h:, h:]
    C1, C2, C3 = C[:h, :h], C[:h, h:], C[h:, h:]
    X1 = trss(U1, C1, p, mistake)
    D2 = _mod(C2 - _mm(X1.T, U2, p), p)
    X2 = _upperT_solve(U1, D2, p)
    D3 = _mod(C3 - (_mm(X2.T, U2, p) + _mm(U2.T, X2, p)), p)
    X3 = trss(U3, D3, p, mistake)
    X = _z(n, n)
    X[:h, :h] = X1
    X[:h, h:] = X2
    X[h:, h:] = X3
    return X


# ---------------------------------------------------------------------------
# PLDUQ revealing the rank profile matrix (reading G1)
# ---------------------------------------------------------------------------

def plduq(B, p: int):
    """B[prow[i], qcol[j]] == (Lf diag(D) U)[i, j] with Lf (m x r) unit lower
    trapezoidal [L1; M1] and U (r x n) unit upper trapezoidal [U1 V1].

    Rows are taken in order.  Each row is reduced against the pivot rows
    found so far (in their order, each normalised to 1 at its pivot column);
    a non-zero remainder makes the row a pivot row, on the remainder's first
    non-zero column.  So B[i] = sum_k W[i][k] E_k with E_k the normalised
    pivot rows.  Pivot rows keep their order, then the other rows in order;
    pivot columns come in pivot order, then the other columns in order.  The
    pivots (prow[k], qcol[k]) are the leading positions of the echelon form
    built row by row, i.e. the ones of B's rank profile matrix."""
    B = _mod(B, p)
    m, n = B.shape
    E, pcols, prow_piv, dvals = [], [], [], []
    W = {}
    for i in range(m):
        rem = B[i].copy()
        w = []
        for k in range(len(E)):
            c = int(rem[pcols[k]]) % p
            w.append(c)
            if c:
                rem = _mod(rem - c * E[k], p)
        nz = next((j for j in range(n) if int(rem[j]) % p), None)
        if nz is None:
            W[i] = w
            continue
        x = int(rem[nz]) % p
        E.append(_mod(rem * _inv(x, p), p))
        pcols.append(nz)
        prow_piv.append(i)
        dvals.append(x)
        W[i] = w + [x]
    r = len(E)
    prow = prow_piv + [i for i in range(m) if i not in prow_piv]
    qcol = pcols + [j for j in range(n) if j not in pcols]
    Lf = _z(m, r)
    for a, i in enumerate(prow):
        for k, wk in enumerate(W[i]):
            Lf[a, k] = wk * _inv(dvals[k], p) % p
    U = _z(r, n)
    for k in range(r):
        U[k] = np.array([E[k][c] for c in qcol], dtype=object)
    return dict(prow=prow, qcol=qcol, L=Lf, D=dvals, U=U, r=r)


# ---------------------------------------------------------------------------
# Algorithms 2 and 3
# ---------------------------------------------------------------------------

def _result(perm, L, D, p, sort_zero=True):
    """(perm, L, D) -> the result dict.  The non-pivot rows (positions from
    the rank on, where L is [L21 I] and D is zero) are put in ascending
    original order, permuting their L rows alike, which keeps the identity."""
    N = len(perm)
    if sort_zero and N:
        r0 = _rank_of(D, p)
        order = sorted(range(r0, N), key=lambda k: perm[k])
        if order != list(range(r0, N)):
            perm = list(perm[:r0]) + [perm[k] for k in order]
            L = L.copy()
            L[r0:, :r0] = L[order, :r0]
    N = len(perm)
    d = [int(D[k, k]) % p for k in range(N)]
    e = [0] * N
    k = 0
    rank = 0
    while k < N:
        if k + 1 < N and int(D[k + 1, k]) % p:
            e[k] = int(D[k + 1, k]) % p
            rank += 2
            k += 2
        else:
            if d[k]:
                rank += 1
            k += 1
    return dict(perm=list(perm), L=L, D=D, d=d, e=e, rank=rank)


def _rank_of(D, p):
    N = D.shape[0]
    k = r = 0
    while k < N:
        if k + 1 < N and int(D[k + 1, k]) % p:
            r, k = k + 2, k + 2
        else:
            if int(D[k, k]) % p:
                r = k + 1
            k += 1
    return r


def ldlt_alg2(M, p: int, base: int = 1, mistake: str = "none"):
    """Algorithm 2 on the symmetric N x N matrix M (full symmetric storage).
    Returns dict(perm, L, D, d, e, rank) with P^T M P = L D L^T, P e_k =
    e_perm[k], pivots first (rank of them), zero rows last.  Sizes N <= base
    use Algorithm 4 (the cascade of Section 6)."""
    M = _mod(M, p)
    N = M.shape[0]
    if N == 0:
        return _result([], _z(0, 0), _z(0, 0), p)
    if N <= base and N > 1:
        return _alg4(M, p)
    if N == 1:
        L = np.array([[1]], dtype=object)
        D = np.array([[int(M[0, 0]) % p]], dtype=object)
        return _result([0], L, D, p)
    m = N // 2
    n = N - m
    A, B, C = M[:m, :m], M[:m, m:], M[m:, m:]
    fa = ldlt_alg2(A, p, base, mistake)
    r = fa["rank"]
    P1 = fa["perm"]
    L1 = fa["L"][:r, :r]
    M1 = fa["L"][r:, :r]
    D1 = fa["D"][:r, :r]
    Bp = B[P1, :]                                  # PERM(P1^T, B)
    X = _lower_solve(L1, Bp[:r], p) if r else _z(0, n)          # TRSM
    Y = _mod(Bp[r:] - _mm(M1, X, p), p)            # GEMM
    D1inv = _block_inverse(D1, p)
    G = _mm(X.T, D1inv, p) if r else _z(n, 0)      # SCAL by D1^{-1}
    sign = 1 if mistake == "z_plus" else -1
    Z = _mod(C + sign * _mm(_mm(G, D1, p), G.T, p), p) if r else C.copy()   # SYRDK
    f2 = ldlt_alg3(Y, Z, p, base, mistake)         # [[0, Y], [Y^T, Z]]
    P2 = f2["perm"]
    sub = P1[r:] + [m + j for j in range(n)]       # indices of the Algorithm 3 block
    perm = P1[:r] + [sub[i] for i in P2]
    N1 = np.concatenate([M1, G], axis=0)[P2, :] if r else _z(N - r, 0)
    L = _z(N, N)
    D = _z(N, N)
    L[:r, :r] = L1
    L[r:, :r] = N1
    L[r:, r:] = f2["L"]
    D[:r, :r] = D1
    D[r:, r:] = f2["D"]
    return _result(perm, L, D, p)


def ldlt_alg3(Bm, C, p: int, base: int = 1, mistake: str = "none"):
    """Algorithm 3 on [[0, Bm], [Bm^T, C]] (Bm m x n, C n x n symmetric).
    Indices 0..m-1 are Bm's rows, m..m+n-1 C's."""
    Bm = _mod(Bm, p)
    C = _mod(C, p)
    m, n = Bm.shape[0], C.shape[0]
    if m == 0:
        return ldlt_alg2(C, p, base, mistake)
    if n == 0:
        return _result(list(range(m)), _identity(m), _z(m, m), p)
    f = plduq(Bm, p)
    r = f["r"]
    prow, qcol = f["prow"], f["qcol"]
    if r == 0:
        fz = ldlt_alg2(C, p, base, mistake)
        perm = [m + j for j in fz["perm"]] + list(range(m))
        L = _z(m + n, m + n)
        D = _z(m + n, m + n)
        L[:n, :n] = fz["L"]
        L[n:, n:] = _identity(m)
        D[:n, :n] = fz["D"]
        return _result(perm, L, D, p)
    L1f, Uf, D1v = f["L"], f["U"], f["D"]
    M1 = L1f[r:, :]
    U1, V1 = Uf[:, :r], Uf[:, r:]
    D1 = _diag(D1v)
    D1inv = _diag([_inv(v, p) for v in D1v])
    Cq = C[np.ix_(qcol, qcol)]                     # PERM: C' = Q C Q^T
    C1, C2, C3 = Cq[:r, :r], Cq[:r, r:], Cq[r:, r:]
    Delta = _z(r, r)
    if p == 2 and mistake != "no_delta":
        for i in range(r):
            s = int(C1[i, i])
            for j in range(i):
                s -= int(Delta[j, j]) * int(U1[j, i]) ** 2
            Delta[i, i] = s % p
        C1 = _mod(C1 - _mm(_mm(U1.T, Delta, p), U1, p), p)   # SYRDK
    if p == 2 and mistake == "no_delta":
        C1 = C1.copy()
        for i in range(r):
            C1[i, i] = 0
    X = trss(U1, C1, p, mistake)                   # TRSS
    G1 = _mm(X.T, D1inv, p)                        # SCAL
    if p == 2:
        X = _mod(X + _mm(Delta, U1, p), p)         # DADD
    C2b = _mod(C2 - _mm(X.T, V1, p), p)            # TRMM
    Yb = _upperT_solve(U1, C2b, p)                 # TRSM
    Z = _mod(C3 - (_mm(Yb.T, V1, p) + _mm(V1.T, Yb, p)), p)   # SYRD2K
    if p == 2:
        Z = _mod(Z - _mm(_mm(V1.T, Delta, p), V1, p), p)      # SYRDK
    G2 = _mm(Yb.T, D1inv, p)                       # SCAL
    f3 = ldlt_alg2(Z, p, base, mistake)
    P3 = f3["perm"]
    nr = n - r
    N = m + n
    # final order: interleaved (B pivot row k, C pivot column k), then Z's
    # order, then Bm's non-pivot rows
    perm = []
    for k in range(r):
        perm += [prow[k], m + qcol[k]]
    perm += [m + qcol[r + i] for i in P3]
    perm += prow[r:]
    L = _z(N, N)
    D = _z(N, N)
    interleave = mistake != "no_interleave"
    c1 = (lambda k: 2 * k) if interleave else (lambda k: k)
    c2 = (lambda k: 2 * k + 1) if interleave else (lambda k: r + k)
    rb = c1 if interleave else (lambda k: k)        # row of B pivot row k
    rc = c2 if interleave else (lambda k: r + k)    # row of C pivot column k
    if not interleave:
        perm = [prow[k] for k in range(r)] + [m + qcol[k] for k in range(r)] + perm[2 * r:]
    for i in range(r):
        for k in range(r):
            L[rb(i), c1(k)] = L1f[i, k]
            L[rc(i), c1(k)] = G1[i, k]
            L[rc(i), c2(k)] = U1[k, i]
        D[rb(i), c2(i)] = D1v[i]
        D[rc(i), c1(i)] = D1v[i]
        D[rc(i), c2(i)] = Delta[i, i]
    for a, zi in enumerate(P3):                    # rows of the Z part, in P3 order
        row = 2 * r + a
        for k in range(r):
            L[row, c1(k)] = G2[zi, k]
            L[row, c2(k)] = V1[k, zi]
    L[2 * r:2 * r + nr, 2 * r:2 * r + nr] = f3["L"]
    D[2 * r:2 * r + nr, 2 * r:2 * r + nr] = f3["D"]
    for a in range(m - r):                         # Bm's non-pivot rows, last
        row = 2 * r + nr + a
        for k in range(r):
            L[row, c1(k)] = M1[a, k]
        L[row, row] = 1
    return _result(perm, L, D, p)


def _identity(n):
    I = _z(n, n)
    for i in range(n):
        I[i, i] = 1
    return I


def _diag(v):
    D = _z(len(v), len(v))
    for i, x in enumerate(v):
        D[i, i] = x
    return D


def _block_inverse(D, p):
    """Inverse of a block diagonal D with 1x1 blocks and 2x2 blocks
    [[0, x], [x, y]] (the 2x2 blocks are found from the subdiagonal)."""
    n = D.shape[0]
    R = _z(n, n)
    k = 0
    while k < n:
        if k + 1 < n and int(D[k + 1, k]) % p:
            a, b, c = int(D[k, k]), int(D[k, k + 1]), int(D[k + 1, k + 1])
            det = (a * c - b * b) % p
            di = _inv(det, p)
            R[k, k] = c * di % p
            R[k, k + 1] = (-b) * di % p
            R[k + 1, k] = (-b) * di % p
            R[k + 1, k + 1] = a * di % p
            k += 2
        else:
            R[k, k] = _inv(D[k, k], p)
            k += 1
    return R


def _alg4(M, p):
    """Algorithm 4 (the C oracle) as the base case of the cascade."""
    from . import oracle as o
    N = M.shape[0]
    A = np.array([[int(M[i, j]) % p for j in range(N)] for i in range(N)], dtype=np.int64)
    f = o.ldlt_rpm(np.tril(A).astype(np.uint32), p)
    L = np.array(f["L"].astype(np.int64), dtype=object)
    D = np.array(o.build_D(f["d"], f["e"], p), dtype=object)
    return _result([int(v) for v in f["perm"]], L, D, p)


# ---------------------------------------------------------------------------
# given-P mode
# ---------------------------------------------------------------------------

def factor_given_p(A, perm, starts, rank: int, p: int):
    """The L and D of P^T A P = L D L^T for the pivot order `perm` (P e_k =
    e_perm[k]), 2x2 block starts `starts` (bool per position) and `rank`
    pivot positions; A is read as a full symmetric matrix.

    Plain right-looking block elimination of S = P^T A P: a 1x1 pivot needs
    S_kk != 0; a 2x2 block (k, k+1) needs S_kk = 0 and x = S_k+1,k != 0, takes
    D = [[0, x], [x, 0]] and in-block l = y / (2x) (odd p) or D = [[0, x],
    [x, y]] and l = 0 (p = 2), y = S_k+1,k+1; after `rank` positions the
    Schur complement must vanish.  Raises ValueError when the structure does
    not fit A.  For odd p the result is unique (a 2x2 block [[0, x], [x, y]]
    = [[1, 0], [l, 1]] [[0, x], [x, 0]] [[1, l], [0, 1]] forces l = y / (2x)),
    so any algorithm producing this P and block structure gives this L, D."""
    A = _mod(A, p)
    N = A.shape[0]
    S = A[np.ix_(perm, perm)].copy()
    L = _identity(N)
    D = _z(N, N)
    k = 0
    while k < rank:
        if starts[k]:
            if k + 1 >= rank:
                raise ValueError("2x2 block past the rank")
            if int(S[k, k]) % p:
                raise ValueError("2x2 block with a non-zero leading entry at %d" % k)
            x, y = int(S[k + 1, k]) % p, int(S[k + 1, k + 1]) % p
            if x == 0:
                raise ValueError("singular 2x2 block at %d" % k)
            if p == 2:
                ell, Db = 0, np.array([[0, x], [x, y]], dtype=object)
            else:
                ell, Db = y * _inv(2 * x, p) % p, np.array([[0, x], [x, 0]], dtype=object)
            Lb = np.array([[1, 0], [ell, 1]], dtype=object)
            L[k + 1, k] = ell
            D[k:k + 2, k:k + 2] = Db
            Cb = S[k + 2:, k:k + 2]
            # L_below (Db Lb^T) = Cb
            T = _mm(Db, Lb.T, p)
            det = (int(T[0, 0]) * int(T[1, 1]) - int(T[0, 1]) * int(T[1, 0])) % p
            di = _inv(det, p)
            Ti = np.array([[T[1, 1] * di % p, (-T[0, 1]) * di % p],
                           [(-T[1, 0]) * di % p, T[0, 0] * di % p]], dtype=object)
            Lbelow = _mm(Cb, Ti, p)
            L[k + 2:, k:k + 2] = Lbelow
            Mi = _inv2(S[k:k + 2, k:k + 2], p)
            S[k + 2:, k + 2:] = _mod(S[k + 2:, k + 2:] - _mm(_mm(Cb, Mi, p), Cb.T, p), p)
            k += 2
        else:
            dk = int(S[k, k]) % p
            if dk == 0:
                raise ValueError("zero 1x1 pivot at %d" % k)
            D[k, k] = dk
            col = _mod(S[k + 1:, k] * _inv(dk, p), p)
            L[k + 1:, k] = col
            S[k + 1:, k + 1:] = _mod(S[k + 1:, k + 1:] - dk * np.outer(col, col), p)
            k += 1
    if k != rank:
        raise ValueError("block structure does not end at the rank")
    if any(int(v) % p for v in S[rank:, rank:].ravel()):
        raise ValueError("Schur complement beyond the rank is not zero")
    return _result(list(perm), L, D, p)


def _inv2(Mb, p):
    a, b, c, d = (int(Mb[0, 0]), int(Mb[0, 1]), int(Mb[1, 0]), int(Mb[1, 1]))
    det = (a * d - b * c) % p
    di = _inv(det, p)
    return np.array([[d * di % p, (-b) * di % p], [(-c) * di % p, a * di % p]], dtype=object)


# ---------------------------------------------------------------------------
# checks
# ---------------------------------------------------------------------------

def check_identity(A, res, p: int) -> bool:
    """P^T A P == L D L^T exactly, L unit lower triangular."""
    A = _mod(A, p)
    perm = res["perm"]
    L, D = res["L"], res["D"]
    N = A.shape[0]
    for i in range(N):
        if int(L[i, i]) % p != 1 or any(int(L[i, j]) % p for j in range(i + 1, N)):
            return False
    lhs = A[np.ix_(perm, perm)]
    rhs = _mm(_mm(L, D, p), L.T, p)
    return all(int(a) % p == int(b) % p for a, b in zip(lhs.ravel(), rhs.ravel()))


def rpm_matrix(res, N):
    """P Psi P^T from the (perm, block) structure: 1x1 pivot k gives
    R[perm[k], perm[k]] = 1, a 2x2 block (k, k+1) gives R[perm[k], perm[k+1]]
    = R[perm[k+1], perm[k]] = 1 (Section 2.1)."""
    R = np.zeros((N, N), dtype=np.int64)
    perm, e, d = res["perm"], res["e"], res["d"]
    k = 0
    while k < N:
        if e[k]:
            a, b = perm[k], perm[k + 1]
            R[a, b] = R[b, a] = 1
            k += 2
        else:
            if d[k]:
                R[perm[k], perm[k]] = 1
            k += 1
    return R
