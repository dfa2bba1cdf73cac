"""The identity the tensor-core TRSS step rests on, checked on the CPU against
the oracle's Algorithm 1 (Section 4, Problem 1).

For U upper triangular with a non-zero diagonal and V = U^{-1}, the solution
X of X^T U + U^T X = C gives M = X V upper triangular with
M + M^T = V^T C V =: S.  So M is S's strict upper triangle plus half its
diagonal (p = 2: a zero diagonal, which is x_ii = 0, and S must have a zero
diagonal), X = M U, and a block row of the solution is
X_12 = V_1^T (C_12 - X_11^T U_12).  The GPU step computes X_kk and the panel
this way instead of by substitution; these checks tie that reading to the
recursive oracle's X, which the oracle pins pin to the paper."""
import numpy as np
import pytest

from oracle import oracle as o
from oracle import recursive as rc


def _upper_inverse(U, p):
    """V with V U = I for U upper triangular mod p, row by row (textbook
    back substitution: v_ii = 1/u_ii, v_il = -(sum_{i<=k<l} v_ik u_kl)/u_ll)."""
    n = U.shape[0]
    V = [[0] * n for _ in range(n)]
    for i in range(n):
        V[i][i] = pow(int(U[i, i]), -1, p)
        for l in range(i + 1, n):
            s = sum(V[i][k] * int(U[k, l]) for k in range(i, l)) % p
            V[i][l] = (-s * pow(int(U[l, l]), -1, p)) % p
    return np.array(V, dtype=np.int64)


def _inputs(n, p, seed):
    rng = np.random.default_rng(seed)
    hi = min(p, 1 << 31)
    U = np.triu(rng.integers(0, hi, size=(n, n), dtype=np.int64)) % p
    for i in range(n):
        U[i, i] = int(rng.integers(1, p)) if p > 2 else 1
    if p == 2:  # a consistent right-hand side: C = Y^T U + U^T Y
        Y = np.triu(rng.integers(0, 2, size=(n, n)))
        C = (o.matmul_mod(Y.T, U, 2) + o.matmul_mod(U.T, Y, 2)) % 2
    else:
        C = rng.integers(0, hi, size=(n, n), dtype=np.int64) % p
        C = np.triu(C) + np.triu(C, 1).T
    return U, C


@pytest.mark.parametrize("p", [2, 3, 65521, 8388593, 2147483647])
@pytest.mark.parametrize("n", [1, 6, 17, 40])
def test_trss_solution_through_the_inverse(p, n):
    U, C = _inputs(n, p, 7 * n + p % 89)
    X = np.array(rc.trss(U, C, p), dtype=np.int64)
    V = _upper_inverse(U, p)
    assert np.array_equal(o.matmul_mod(V, U, p), np.eye(n, dtype=np.int64))
    M = o.matmul_mod(X, V, p)
    assert not np.any(np.tril(M, -1))  # upper triangular
    S = o.matmul_mod(o.matmul_mod(V.T, C, p), V, p)
    assert np.array_equal((M + M.T) % p, S)
    # M from S alone: strict upper triangle, half the diagonal (p = 2: zero)
    half = 0 if p == 2 else (p + 1) // 2
    Ms = np.triu(S, 1) + np.diag((np.diag(S) * half) % p)
    assert np.array_equal(Ms, M)
    if p == 2:
        assert not np.any(np.diag(S))
    assert np.array_equal(o.matmul_mod(Ms, U, p), X)


@pytest.mark.parametrize("p", [3, 65521, 2147483647])
def test_trss_panel_through_the_inverse(p):
    n, b = 40, 16
    U, C = _inputs(n, p, 99 + p % 13)
    X = np.array(rc.trss(U, C, p), dtype=np.int64)
    V1 = _upper_inverse(U[:b, :b], p)
    T = (C[:b, b:] - o.matmul_mod(X[:b, :b].T, U[:b, b:], p)) % p
    assert np.array_equal(o.matmul_mod(V1.T, T, p), X[:b, b:])


def test_inconsistent_characteristic_2_shows_in_s():
    """p = 2 with a non-zero diagonal entry in C: no X exists, and S = V^T C V
    has a non-zero diagonal entry (the case the GPU step reports)."""
    n = 9
    U, C = _inputs(n, 2, 5)
    C = C.copy()
    C[4, 4] = 1
    V = _upper_inverse(U, 2)
    S = o.matmul_mod(o.matmul_mod(V.T, C, 2), V, 2)
    assert np.any(np.diag(S))
    with pytest.raises(ValueError):
        rc.trss(U, C, 2)
