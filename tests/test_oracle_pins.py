"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Every check here is independent of the oracle's own code path:
* Theorem 1 (Section 2.1): the rank profile matrix is the rook placement whose
  leading blocks have the ranks of A's -- computed by brute force.
* Definition 2 (Section 2.1): the factorisation reveals R_A when
  P Psi P^T = R_A.
* The abstract's identity P^T A P = L D L^T, checked exactly mod p.
* Lemma 1: R_A of a symmetric matrix is symmetric.
* Lemma 2 and the relaxed blocks of Section 2.2 (characteristic 2).
* Planted inputs A = T R T^T: lower-triangular congruence preserves the rank
  of every leading block, so R_A = supp(R).
* A closed form for planted inputs whose pairs do not cross (derived from the
  uniqueness of L and D once P and the block structure are fixed).
* Generic rank profile: the result is textbook unpivoted LDL^T (P = I).
"""
import itertools
import os

import numpy as np
import pytest

from oracle import oracle as o
from paper_1802_10453_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.txt")


def _parse_mat(s):
    return np.array([[int(v) for v in row.split()] for row in s.split(";")], dtype=np.int64)


def _parse_vec(s):
    return np.array([int(v) for v in s.split()], dtype=np.int64)


def _golden():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, p, A, perm, L, d, e, rpm = [x.strip() for x in line.split("|")]
            out.append((name, int(p), _parse_mat(A), _parse_vec(perm), _parse_mat(L),
                        _parse_vec(d), _parse_vec(e), _parse_vec(rpm)))
    return out


def structure_ok(res, p):
    """L unit lower triangular with identity columns beyond the rank; D blocks
    1x1 non-zero, or [[0,x],[x,0]] (odd p) / [[0,x],[x,y]] (p = 2) with x != 0;
    D zero beyond the rank."""
    L, d, e, r = res["L"].astype(np.int64), res["d"], res["e"], res["rank"]
    n = L.shape[0]
    if not np.array_equal(np.diag(L), np.ones(n)):
        return False
    if np.triu(L, 1).any():
        return False
    if n > r and not np.array_equal(L[r:, r:], np.eye(n - r, dtype=np.int64)):
        return False
    k = 0
    while k < r:
        if e[k] != 0:
            if k + 1 >= r or d[k] != 0 or e[k + 1] != 0:
                return False
            if p != 2 and d[k + 1] != 0:
                return False
            k += 2
        else:
            if d[k] == 0:
                return False
            k += 1
    if np.any(d[r:] != 0) or np.any(e[r:] != 0):
        return False
    return True


def full_check(A, p, res=None):
    A = np.asarray(A, dtype=np.int64) % p
    if res is None:
        res = o.ldlt_rpm(A.astype(np.uint32), p)
    assert structure_ok(res, p)
    assert o.check_factor(A, res["perm"], res["L"], res["d"], res["e"], p)
    R = o.rank_profile_bruteforce(A, p)
    assert np.array_equal(R, R.T)                       # Lemma 1
    rpm = o.rpm_from_factor(res["perm"], res["e"], res["rank"])
    assert np.array_equal(o.rpm_col_to_matrix(rpm), R)  # Definition 2: reveals R_A
    perm_c, _ = o.canonical_perm_from_rpm(R)
    assert np.array_equal(res["perm"], perm_c)          # lexicographic order of Algorithm 4
    assert res["rank"] == int(R.sum())
    return res


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c[0])
def test_worked_examples(case):
    name, p, A, perm, L, d, e, rpm = case
    res = o.ldlt_rpm(A.astype(np.uint32), p)
    assert np.array_equal(res["perm"], perm)
    assert np.array_equal(res["L"].astype(np.int64), L)
    assert np.array_equal(res["d"].astype(np.int64), d)
    assert np.array_equal(res["e"].astype(np.int64), e)
    assert np.array_equal(o.rpm_from_factor(res["perm"], res["e"], res["rank"]), rpm)
    full_check(A, p, res)


def test_lemma2_no_strict_factor_in_char2():
    """Lemma 2: over F_2 no L Dbar (diagonal or antidiagonal support) with
    P, Psi in {I, J} reproduces [[0,1],[1,1]] while revealing R_A = J.  This is
    why D needs the relaxed block [[0,c],[c,d]] in characteristic 2."""
    A = np.array([[0, 1], [1, 1]])
    I = np.eye(2, dtype=np.int64)
    J = np.array([[0, 1], [1, 0]])
    found = False
    for x, y, z in itertools.product(range(2), repeat=3):
        Lm = np.array([[1, 0], [x, 1]])
        Db = np.array([[y, 0], [0, z]])
        for P in (I, J):
            for Psi in (I, J):
                D = Psi @ Db
                if not np.array_equal(D % 2, D.T % 2):
                    continue
                M = (P @ Lm @ D @ Lm.T @ P.T) % 2
                if np.array_equal(M, A) and np.array_equal(P @ Psi @ P.T, J):
                    found = True
    assert not found
    res = o.ldlt_rpm(A.astype(np.uint32), 2)
    assert res["d"][1] == 1 and res["e"][0] == 1  # the relaxed block
    full_check(A, 2, res)


def _all_symmetric(n, p):
    idx = [(i, j) for i in range(n) for j in range(i + 1)]
    for vals in itertools.product(range(p), repeat=len(idx)):
        A = np.zeros((n, n), dtype=np.int64)
        for (i, j), v in zip(idx, vals):
            A[i, j] = A[j, i] = v
        yield A


@pytest.mark.parametrize("n,p", [(2, 2), (3, 2), (4, 2), (2, 3), (3, 3), (2, 5)])
def test_exhaustive_small_fields(n, p):
    for A in _all_symmetric(n, p):
        full_check(A, p)


@pytest.mark.parametrize("p", [2, 3, 5, 7, 65521, 2147483647])
def test_random_small_vs_bruteforce(p):
    rng = np.random.default_rng(p)
    for trial in range(25):
        n = int(rng.integers(1, 13))
        kind = trial % 3
        if kind == 0:  # dense uniform symmetric
            B = rng.integers(0, p, size=(n, n))
            A = np.tril(B) + np.tril(B, -1).T
        elif kind == 1:  # sparse symmetric: many zero pivots and 2x2 blocks
            B = rng.integers(0, p, size=(n, n)) * (rng.random((n, n)) < 0.25)
            A = np.tril(B) + np.tril(B, -1).T
        else:  # low rank symmetric
            k = int(rng.integers(0, n + 1))
            X = rng.integers(0, p, size=(n, k))
            A = o.matmul_mod(X, X.T, p) if k else np.zeros((n, n), dtype=np.int64)
        full_check(A % p, p)


@pytest.mark.parametrize("p", [2, 3, 65521, 2147483647])
def test_planted_rank_profile(p):
    """A = T R T^T: R_A = supp(R) (leading blocks of A are T11 R T11^T)."""
    for seed in range(6):
        n = 10 + seed
        r = min(n, 4 + 2 * seed)
        npairs = r // 4 if seed % 2 else r // 2
        A, partner, scale = inputs.planted_matrix(n, r, npairs, p, seed)
        res = full_check(A, p)
        assert np.array_equal(o.rpm_from_factor(res["perm"], res["e"], res["rank"]), partner)


def _noncrossing_plant(n, p, rng):
    """R whose transpositions pair consecutive support indices (no support
    index strictly between the two members of a pair)."""
    sup = np.sort(rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False))
    R = np.zeros((n, n), dtype=np.int64)
    k = 0
    blocks = []
    while k < len(sup):
        s = int(rng.integers(1, p))
        if k + 1 < len(sup) and rng.random() < 0.5:
            a, b = sup[k], sup[k + 1]
            R[a, b] = R[b, a] = s
            blocks.append((a, b, s))
            k += 2
        else:
            R[sup[k], sup[k]] = s
            blocks.append((sup[k], None, s))
            k += 1
    return sup, R, blocks


@pytest.mark.parametrize("p", [3, 5, 65521, 2147483647])
def test_noncrossing_closed_form(p):
    """For odd p and non-crossing pairs, A = T R T^T factors as
    perm = (support ascending, then the rest ascending), L's first r columns =
    T[perm, support], D = R[support, support].  Proof: P^T T_S is
    [T[S,S]; T[N,S]] with T[S,S] unit lower triangular, and R[S,S] is block
    diagonal with antidiagonal pairs; L and D are unique once P and the block
    structure are fixed.  (The in-block L entry T_ba equals y/(2x) since
    y = 2 x T_ba.)"""
    rng = np.random.default_rng(p + 1)
    for trial in range(8):
        n = int(rng.integers(2, 40))
        T = inputs.T_matrix(n, p, 1000 + trial)
        sup, R, blocks = _noncrossing_plant(n, p, rng)
        A = o.matmul_mod(o.matmul_mod(T, R, p), T.T, p)
        res = o.ldlt_rpm(A.astype(np.uint32), p)
        r = len(sup)
        rest = np.array([i for i in range(n) if i not in set(sup.tolist())], dtype=np.int64)
        perm = np.concatenate([sup, rest]).astype(np.int64)
        assert res["rank"] == r
        assert np.array_equal(res["perm"], perm)
        assert np.array_equal(res["L"][:, :r].astype(np.int64), T[np.ix_(perm, sup)] % p)
        D = o.build_D(res["d"], res["e"], p)
        assert np.array_equal(D[:r, :r], R[np.ix_(sup, sup)] % p)


def test_diagonal_plant_closed_form_char2():
    """R diagonal: the closed form holds in every characteristic."""
    p = 2
    rng = np.random.default_rng(7)
    for trial in range(10):
        n = int(rng.integers(2, 30))
        T = inputs.T_matrix(n, p, 77 + trial)
        sup = np.sort(rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False))
        R = np.zeros((n, n), dtype=np.int64)
        R[sup, sup] = 1
        A = o.matmul_mod(o.matmul_mod(T, R, p), T.T, p)
        res = o.ldlt_rpm(A.astype(np.uint32), p)
        rest = np.array([i for i in range(n) if i not in set(sup.tolist())], dtype=np.int64)
        perm = np.concatenate([sup, rest]).astype(np.int64)
        assert np.array_equal(res["perm"], perm)
        assert np.array_equal(res["L"][:, :len(sup)].astype(np.int64), T[np.ix_(perm, sup)] % p)


def _textbook_ldlt(A, p):
    """Unpivoted LDL^T (Golub & Van Loan, Alg. 4.1.2 restated mod p)."""
    n = A.shape[0]
    A = [[int(v) % p for v in row] for row in A]
    L = [[0] * n for _ in range(n)]
    d = [0] * n
    for j in range(n):
        s = A[j][j]
        for k in range(j):
            s -= L[j][k] * L[j][k] * d[k]
        d[j] = s % p
        assert d[j] != 0, "not generic"
        inv = pow(d[j], p - 2, p)
        L[j][j] = 1
        for i in range(j + 1, n):
            s = A[i][j]
            for k in range(j):
                s -= L[i][k] * L[j][k] * d[k]
            L[i][j] = (s % p) * inv % p
    return np.array(L, dtype=np.int64), np.array(d, dtype=np.int64)


@pytest.mark.parametrize("p", [65521, 8388593, 2147483647])
def test_generic_rank_profile_is_textbook_ldlt(p):
    for seed in range(3):
        A = inputs.uniform_symmetric(24, p, seed).astype(np.int64)
        Lt, dt = _textbook_ldlt(A, p)
        res = o.ldlt_rpm(A.astype(np.uint32), p)
        assert np.array_equal(res["perm"], np.arange(24))
        assert np.array_equal(res["L"].astype(np.int64), Lt)
        assert np.array_equal(res["d"].astype(np.int64), dt)
        assert not res["e"].any()


@pytest.mark.parametrize("p", [5, 65521])
def test_scaling_metamorphic(p):
    """c*A = P L (cD) L^T P^T: same perm and L, D scaled by c."""
    rng = np.random.default_rng(3)
    for trial in range(6):
        A, _, _ = inputs.planted_matrix(14, 10, 3, p, 50 + trial)
        c = int(rng.integers(2, p))
        r1 = o.ldlt_rpm(A, p)
        r2 = o.ldlt_rpm(((A.astype(np.int64) * c) % p).astype(np.uint32), p)
        assert np.array_equal(r1["perm"], r2["perm"])
        assert np.array_equal(r1["L"], r2["L"])
        assert np.array_equal((r1["d"].astype(np.int64) * c) % p, r2["d"].astype(np.int64))
        assert np.array_equal((r1["e"].astype(np.int64) * c) % p, r2["e"].astype(np.int64))


def test_config0_size_planted():
    """n = 256, r = 192, p = 65521 planted: exact factor identity and R_A = supp(R)."""
    n, r, p = 256, 192, 65521
    A, partner, _ = inputs.planted_matrix(n, r, r // 4, p, inputs.SEED_BASE)
    res = o.ldlt_rpm(A, p)
    assert res["rank"] == r
    assert o.check_factor(A, res["perm"], res["L"], res["d"], res["e"], p)
    assert np.array_equal(o.rpm_from_factor(res["perm"], res["e"], res["rank"]), partner)
    perm_c, _ = o.canonical_perm_from_rpm(o.rpm_col_to_matrix(partner))
    assert np.array_equal(res["perm"], perm_c)
    assert o.freivalds_check(A, res["perm"], res["L"], res["d"], res["e"], p)


def test_freivalds_detects_error():
    n, r, p = 64, 48, 65521
    A, _, _ = inputs.planted_matrix(n, r, r // 4, p, 5)
    res = o.ldlt_rpm(A, p)
    assert o.freivalds_check(A, res["perm"], res["L"], res["d"], res["e"], p)
    L = res["L"].copy()
    L[40, 3] = (int(L[40, 3]) + 1) % p
    assert not o.freivalds_check(A, res["perm"], L, res["d"], res["e"], p)


def _pins_pass(A, p, mutation):
    A = np.asarray(A, dtype=np.int64) % p
    res = o.ldlt_rpm(A.astype(np.uint32), p, mutation=mutation)
    try:
        full_check(A, p, res)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mutation", [m for m in o.MUTATIONS if m != "none"])
def test_planted_mistakes_are_caught(mutation):
    """Each deliberate mistake planted in the oracle fails at least one pin."""
    caught = False
    for p in (2, 3, 7, 65521):
        for seed in range(6):
            A, _, _ = inputs.planted_matrix(9, 8, 2 + seed % 2, p, 300 + seed)
            if not _pins_pass(A, p, mutation):
                caught = True
                break
        if caught:
            break
    assert caught, mutation
    assert _pins_pass(inputs.planted_matrix(9, 8, 2, 7, 300)[0], 7, "none")


# ---- Section 2.2: antitriangular -> strict factorisation in characteristic 2 ----
def _all_symmetric_f2(n):
    idx = [(i, j) for i in range(n) for j in range(i + 1)]
    for bits in range(1 << len(idx)):
        A = np.zeros((n, n), dtype=np.int64)
        for q, (i, j) in enumerate(idx):
            if bits >> q & 1:
                A[i, j] = A[j, i] = 1
        yield A


def _strict_shape_ok(d, e):
    # only 1x1 pivots and antidiagonal blocks [[0, c], [c, 0]] remain
    for k in range(len(d) - 1):
        if e[k] != 0 and (d[k] != 0 or d[k + 1] != 0):
            return False
    return True


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_char2_strict_transform_exhaustive(n):
    relaxed = 0
    for A in _all_symmetric_f2(n):
        f = o.ldlt_rpm(A.astype(np.uint32), 2)
        if any(f["e"][k] and f["d"][k + 1] for k in range(n - 1)):
            relaxed += 1
        perm, L, d, e = o.strict_char2(f["perm"], f["L"], f["d"], f["e"])
        assert o.check_factor(A, perm, L, d, e, 2)
        assert np.array_equal(np.triu(L, 1), np.zeros_like(L)) and np.all(np.diag(L) == 1)
        assert _strict_shape_ok(d, e)
        assert int(np.count_nonzero(d)) + 2 * int(np.count_nonzero(e)) == f["rank"]
    assert relaxed > 0 or n < 2  # the relaxed blocks of Section 2.2 do occur


def test_char2_strict_worked_example():
    # [[0, 1], [1, 1]] over F_2: P = I, L = I, D = A; strict form P = J,
    # L = [[1, 0], [1, 1]], D = diag(1, 1)
    A = np.array([[0, 1], [1, 1]])
    f = o.ldlt_rpm(A.astype(np.uint32), 2)
    assert list(f["perm"]) == [0, 1] and f["e"][0] == 1 and f["d"][1] == 1
    perm, L, d, e = o.strict_char2(f["perm"], f["L"], f["d"], f["e"])
    assert list(perm) == [1, 0]
    assert np.array_equal(L, [[1, 0], [1, 1]])
    assert list(d) == [1, 1] and list(e) == [0, 0]


def test_char2_strict_odd_p_unchanged():
    A, _, _ = inputs.planted_matrix(40, 30, 8, 7, 3)
    f = o.ldlt_rpm(A, 7)
    perm, L, d, e = o.strict_char2(f["perm"], f["L"], f["d"], f["e"], p=7)
    assert np.array_equal(perm, f["perm"]) and np.array_equal(L, f["L"]) and np.array_equal(e, f["e"])


@pytest.mark.parametrize("mistake", ["no_row_swap", "no_perm_swap", "no_column_op"])
def test_char2_strict_planted_mistakes_fail(mistake):
    caught = False
    for A in _all_symmetric_f2(4):
        f = o.ldlt_rpm(A.astype(np.uint32), 2)
        perm, L, d, e = o.strict_char2(f["perm"], f["L"], f["d"], f["e"], mistake=mistake)
        if not o.check_factor(A, perm, L, d, e, 2):
            caught = True
            break
    assert caught


# ---- consumer: A X = B from the factorisation ----
@pytest.mark.parametrize("p", [2, 3, 65521, 2147483647])
def test_solve_full_rank_is_exact(p):
    rng = np.random.default_rng(p % 1000)
    for n in (1, 2, 7, 40):
        A, _, _ = inputs.planted_matrix(n, n, n // 4, p, 100 + n)
        f = o.ldlt_rpm(A, p)
        assert f["rank"] == n
        B = rng.integers(0, p, size=(n, 3), dtype=np.int64)
        X, ok = o.solve_factor(f["perm"], f["L"], f["d"], f["e"], f["rank"], B, p)
        assert ok
        S = o.symmetrize_lower(A, p)
        assert np.array_equal(o.matmul_mod(S, X, p), B % p)
        # unique solution: agrees with Gaussian elimination's answer on one column
        Ainv_b = _gauss_solve(S, B[:, 0], p)
        assert np.array_equal(X[:, 0], Ainv_b)


def _gauss_solve(S, b, p):
    """Plain Gauss-Jordan elimination mod p for a non-singular S (textbook)."""
    n = S.shape[0]
    M = np.concatenate([S % p, (b % p)[:, None]], axis=1).astype(object)
    for c in range(n):
        piv = next(i for i in range(c, n) if M[i, c] % p)
        M[[c, piv]] = M[[piv, c]]
        M[c] = (M[c] * o.inv_mod(int(M[c, c]), p)) % p
        for i in range(n):
            if i != c and M[i, c] % p:
                M[i] = (M[i] - M[i, c] * M[c]) % p
    return np.array([int(v) for v in M[:, n]], dtype=np.int64)


@pytest.mark.parametrize("p", [2, 7, 65521])
def test_solve_singular_consistency(p):
    rng = np.random.default_rng(7 + p)
    n, r = 30, 18
    A, _, _ = inputs.planted_matrix(n, r, r // 4, p, 55)
    S = o.symmetrize_lower(A, p)
    f = o.ldlt_rpm(A, p)
    assert f["rank"] == r
    # B in the column space: B = S Y for a random Y
    Yr = rng.integers(0, p, size=(n, 2), dtype=np.int64)
    B = o.matmul_mod(S, Yr, p)
    X, ok = o.solve_factor(f["perm"], f["L"], f["d"], f["e"], f["rank"], B, p)
    assert ok and np.array_equal(o.matmul_mod(S, X, p), B)
    # a right-hand side outside the column space is reported
    found = False
    for trial in range(20):
        b = rng.integers(0, p, size=n, dtype=np.int64)
        _, ok = o.solve_factor(f["perm"], f["L"], f["d"], f["e"], f["rank"], b, p)
        in_space = o.rank_mod_p(np.concatenate([S, b[:, None]], axis=1), p) == r
        assert ok == in_space
        found = found or not ok
    assert found
