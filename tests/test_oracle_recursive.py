"""Pins of the recursive oracle (Section 4: Algorithms 1, 2, 3; the given-P
mode), against what the mathematics fixes rather than against itself:

* TRSS: the defining identity X^T U + U^T X = C with X upper triangular, and
  uniqueness by brute force over every upper triangular X on tiny sizes.
* PLDUQ: the factor identity, and its pivots equal to the rank profile matrix
  computed from leading-block ranks (Theorem 1), exhaustively on small F_2
  matrices and randomly elsewhere.
* Algorithms 2/3: P^T A P = L D L^T exactly, D block diagonal of the allowed
  forms, and P Psi P^T equal to the brute-force rank profile matrix
  (Theorem 2), exhaustively for every symmetric matrix over F_2 (n <= 4) and
  F_3 (n <= 3), randomly up to n = 16 and for the cascade with Algorithm 4.
* Given-P mode: on Algorithm 4's pivot order it reproduces the Algorithm 4
  oracle's L and D bit for bit (two unrelated procedures); on the recursion's
  order it reproduces the recursion's L and D (odd p); brute-force uniqueness
  over all unit lower L and block D on F_3, n = 3.
* Planted mistakes (a sign, the halving of TRSS, the interleaving P_i, the
  characteristic-2 Delta) each break one of the checks above.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as o
from oracle import recursive as rc
from paper_1802_10453_gb300 import inputs


def _sym(A, p):
    A = np.asarray(A, dtype=np.int64) % p
    return np.tril(A) + np.tril(A, -1).T


def _obj(A):
    return np.array(np.asarray(A, dtype=np.int64), dtype=object)


def _blocks_valid(res, p):
    """D block diagonal: 1x1 blocks d != 0, 2x2 blocks [[0, x], [x, 0]] (odd p)
    or [[0, x], [x, y]] (p = 2) with x != 0, zero from the rank on."""
    D = np.array(res["D"], dtype=object)
    N = D.shape[0]
    k = 0
    r = res["rank"]
    while k < r:
        if res["e"][k]:
            if int(D[k, k]) % p or int(D[k + 1, k]) % p == 0 or int(D[k, k + 1]) % p != int(D[k + 1, k]) % p:
                return False
            if p != 2 and int(D[k + 1, k + 1]) % p:
                return False
            cols = [c for c in range(N) if c not in (k, k + 1)]
            if any(int(D[k, c]) % p or int(D[k + 1, c]) % p for c in cols):
                return False
            k += 2
        else:
            if int(D[k, k]) % p == 0 or any(int(D[k, c]) % p for c in range(N) if c != k):
                return False
            k += 1
    return not any(int(v) % p for v in D[r:, :].ravel())


# ---------------------------------------------------------------------------
# TRSS (Algorithm 1)
# ---------------------------------------------------------------------------

def _trss_ok(U, C, X, p):
    U = _obj(U)
    lhs = rc._mod(X.T.dot(U) + U.T.dot(X), p)
    upper = all(int(X[i, j]) % p == 0 for i in range(X.shape[0]) for j in range(i))
    return upper and all(int(a) == int(b) % p for a, b in zip(lhs.ravel(), np.asarray(C).ravel()))


@pytest.mark.parametrize("p", [3, 5, 7, 65521, 2147483647])
def test_trss_identity(p):
    rng = np.random.default_rng(p % 1000)
    for n in range(1, 10):
        U = np.triu(rng.integers(0, min(p, 1 << 30), size=(n, n))) % p
        for i in range(n):
            U[i, i] = rng.integers(1, min(p, 1 << 30))
        C = _sym(rng.integers(0, min(p, 1 << 30), size=(n, n)), p)
        assert _trss_ok(U, C, rc.trss(U, C, p), p)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_trss_unique_by_brute_force(n):
    p = 5
    rng = np.random.default_rng(n)
    U = np.triu(rng.integers(0, p, size=(n, n)))
    for i in range(n):
        U[i, i] = rng.integers(1, p)
    C = _sym(rng.integers(0, p, size=(n, n)), p)
    X = rc.trss(U, C, p)
    pos = [(i, j) for i in range(n) for j in range(i, n)]
    sols = []
    for vals in itertools.product(range(p), repeat=len(pos)):
        Y = np.zeros((n, n), dtype=np.int64)
        for (i, j), v in zip(pos, vals):
            Y[i, j] = v
        if np.array_equal((Y.T @ U + U.T @ Y) % p, C):
            sols.append(Y)
    assert len(sols) == 1
    assert np.array_equal(sols[0], np.array(X, dtype=np.int64))


def test_trss_characteristic_2_zero_diagonal():
    rng = np.random.default_rng(2)
    for n in range(1, 9):
        U = np.triu(rng.integers(0, 2, size=(n, n)))
        np.fill_diagonal(U, 1)
        C = _sym(rng.integers(0, 2, size=(n, n)), 2)
        np.fill_diagonal(C, 0)
        assert _trss_ok(U, C, rc.trss(U, C, 2), 2)
    with pytest.raises(ValueError):
        rc.trss(np.eye(1, dtype=np.int64), np.ones((1, 1), dtype=np.int64), 2)


def test_trss_planted_mistake_no_halving():
    U = np.array([[1, 2], [0, 3]])
    C = np.array([[4, 1], [1, 5]])
    assert _trss_ok(U, C, rc.trss(U, C, 7), 7)
    assert not _trss_ok(U, C, rc.trss(U, C, 7, mistake="no_halving"), 7)


# ---------------------------------------------------------------------------
# PLDUQ revealing the rank profile matrix
# ---------------------------------------------------------------------------

def _plduq_ok(B, p):
    f = rc.plduq(B, p)
    m, n = np.asarray(B).shape
    r = f["r"]
    L, U = f["L"], f["U"]
    for k in range(r):  # unit trapezoidal
        if int(L[k, k]) != 1 or int(U[k, k]) != 1:
            return False
        if any(int(L[k, j]) for j in range(k + 1, r)) or any(int(U[k, j]) for j in range(k)):
            return False
    rec = rc._mod(L.dot(rc._diag(f["D"])).dot(U), p) if r else rc._z(m, n)
    Bp = np.asarray(B, dtype=np.int64)[np.ix_(f["prow"], f["qcol"])] % p
    if not all(int(a) == int(b) for a, b in zip(np.asarray(rec).ravel(), Bp.ravel())):
        return False
    R = np.zeros((m, n), dtype=np.int64)
    for k in range(r):
        R[f["prow"][k], f["qcol"][k]] = 1
    return np.array_equal(R, o.rank_profile_bruteforce(B, p))


def test_plduq_exhaustive_f2_2x3():
    for bits in range(1 << 6):
        B = np.array([(bits >> k) & 1 for k in range(6)], dtype=np.int64).reshape(2, 3)
        assert _plduq_ok(B, 2)


@pytest.mark.parametrize("p", [2, 3, 7, 65521])
def test_plduq_random_low_rank(p):
    rng = np.random.default_rng(p)
    for _ in range(60):
        m, n = (int(v) for v in rng.integers(1, 8, size=2))
        r = int(rng.integers(0, min(m, n) + 1))
        B = (rng.integers(0, p, size=(m, r)) @ rng.integers(0, p, size=(r, n))) % p if r else np.zeros((m, n), np.int64)
        assert _plduq_ok(B, p)


# ---------------------------------------------------------------------------
# Algorithms 2 and 3
# ---------------------------------------------------------------------------

def _alg2_ok(S, p, base=1, mistake="none"):
    res = rc.ldlt_alg2(_obj(S), p, base=base, mistake=mistake)
    n = S.shape[0]
    return (rc.check_identity(_obj(S), res, p) and _blocks_valid(res, p)
            and np.array_equal(rc.rpm_matrix(res, n), o.rank_profile_bruteforce(S, p)))


def _all_symmetric(n, p):
    pos = [(i, j) for i in range(n) for j in range(i + 1)]
    for vals in itertools.product(range(p), repeat=len(pos)):
        S = np.zeros((n, n), dtype=np.int64)
        for (i, j), v in zip(pos, vals):
            S[i, j] = S[j, i] = v
        yield S


@pytest.mark.parametrize("n,p", [(1, 2), (2, 2), (3, 2), (4, 2), (1, 3), (2, 3), (3, 3)])
def test_recursive_exhaustive_small_fields(n, p):
    for S in _all_symmetric(n, p):
        assert _alg2_ok(S, p), S


@pytest.mark.parametrize("p", [2, 5, 7, 65521, 2147483647])
@pytest.mark.parametrize("base", [1, 2, 4])
def test_recursive_random_planted(p, base):
    rng = np.random.default_rng(p % 977 + base)
    for t in range(12):
        n = int(rng.integers(2, 17))
        r = int(rng.integers(0, n + 1))
        pairs = [r // 4, r // 2][t % 2]
        A, _, _ = inputs.planted_matrix(n, r, pairs, p, 7000 + 31 * t + base)
        S = _sym(A, p)
        assert _alg2_ok(S, p, base=base)


def test_recursive_uniform_full_rank():
    rng = np.random.default_rng(9)
    for p in (3, 65521):
        for n in (5, 8, 13):
            S = _sym(rng.integers(0, p, size=(n, n)), p)
            assert _alg2_ok(S, p)


def _some_fail(S_list, p, mistake, base=1):
    return any(not _alg2_ok(S, p, base=base, mistake=mistake) for S in S_list)


def test_recursive_planted_mistakes_are_caught():
    rng = np.random.default_rng(13)
    odd = []
    for t in range(20):
        n = int(rng.integers(3, 10))
        A, _, _ = inputs.planted_matrix(n, n - 1, (n - 1) // 2, 7, 900 + t)
        odd.append(_sym(A, 7))
    assert all(_alg2_ok(S, 7) for S in odd)
    for m in ("z_plus", "no_halving", "no_interleave"):
        assert _some_fail(odd, 7, m), m
    two = [S for S in _all_symmetric(3, 2)]
    assert all(_alg2_ok(S, 2) for S in two)
    assert _some_fail(two, 2, "no_delta")


# ---------------------------------------------------------------------------
# given-P mode
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [2, 3, 5, 65521, 2147483647])
def test_given_p_reproduces_algorithm4(p):
    rng = np.random.default_rng(p % 1009)
    for t in range(25):
        n = int(rng.integers(1, 14))
        r = int(rng.integers(0, n + 1))
        A, _, _ = inputs.planted_matrix(n, r, r // 3, p, 300 + t)
        A = np.asarray(A, dtype=np.int64) % p
        f4 = o.ldlt_rpm(np.tril(A).astype(np.uint32), p)
        g = rc.factor_given_p(_obj(_sym(A, p)), [int(v) for v in f4["perm"]], [bool(v) for v in f4["e"]],
                              f4["rank"], p)
        assert np.array_equal(np.array(g["L"], dtype=np.int64), f4["L"].astype(np.int64))
        assert g["d"] == [int(v) for v in f4["d"]] and g["e"] == [int(v) for v in f4["e"]]


@pytest.mark.parametrize("p", [3, 7, 65521])
def test_given_p_reproduces_the_recursion(p):
    rng = np.random.default_rng(p)
    for t in range(20):
        n = int(rng.integers(2, 14))
        r = int(rng.integers(0, n + 1))
        A, _, _ = inputs.planted_matrix(n, r, r // 2, p, 600 + t)
        S = _obj(_sym(A, p))
        rec = rc.ldlt_alg2(S, p)
        g = rc.factor_given_p(S, rec["perm"], [bool(v) for v in rec["e"]], rec["rank"], p)
        assert np.array_equal(np.array(g["L"], dtype=np.int64) % p, np.array(rec["L"], dtype=np.int64) % p)
        assert g["d"] == rec["d"] and g["e"] == rec["e"]


def test_given_p_unique_by_brute_force():
    """F_3, n = 3: every unit lower L and every D of the supplied block
    structure (values of D that the structure does not use give the same
    pair); exactly one pair satisfies the identity."""
    p = 3
    S = np.array([[0, 1, 2], [1, 1, 0], [2, 0, 2]], dtype=np.int64)
    f4 = o.ldlt_rpm(np.tril(S).astype(np.uint32), p)
    perm, starts, r = [int(v) for v in f4["perm"]], [bool(v) for v in f4["e"]], f4["rank"]
    g = rc.factor_given_p(_obj(S), perm, starts, r, p)
    B = S[np.ix_(perm, perm)]
    sols = []
    for l10, l20, l21 in itertools.product(range(p), repeat=3):
        L = np.array([[1, 0, 0], [l10, 1, 0], [l20, l21, 1]], dtype=np.int64)
        for dv in itertools.product(range(p), repeat=3):
            D = np.zeros((3, 3), dtype=np.int64)
            k = 0
            while k < 3:
                if k < r and starts[k]:
                    D[k, k + 1] = D[k + 1, k] = dv[k]
                    if dv[k] == 0:
                        break
                    k += 2
                else:
                    D[k, k] = dv[k] if k < r else 0
                    if k < r and dv[k] == 0:
                        break
                    k += 1
            else:
                if np.array_equal(L @ D @ L.T % p, B):
                    key = (L.tobytes(), D.tobytes())
                    if key not in {(a.tobytes(), b.tobytes()) for a, b in sols}:
                        sols.append((L, D))
    assert len(sols) == 1
    assert np.array_equal(sols[0][0], np.array(g["L"], dtype=np.int64))
    assert np.array_equal(sols[0][1], np.array(g["D"], dtype=np.int64))


def test_given_p_rejects_structures_that_do_not_fit():
    p = 7
    S = _obj(np.array([[0, 1, 0], [1, 2, 0], [0, 0, 3]]))
    with pytest.raises(ValueError):
        rc.factor_given_p(S, [0, 1, 2], [False, False, False], 3, p)     # zero 1x1 pivot
    with pytest.raises(ValueError):
        rc.factor_given_p(S, [2, 0, 1], [True, False, False], 3, p)      # 2x2 block on a non-zero S_kk
    with pytest.raises(ValueError):
        rc.factor_given_p(S, [0, 1, 2], [True, False, False], 2, p)      # rank too small: Schur left over
    g = rc.factor_given_p(S, [0, 1, 2], [True, False, False], 3, p)
    assert rc.check_identity(S, g, p)
