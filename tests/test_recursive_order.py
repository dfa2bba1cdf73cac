"""recursive_order (host logic of the product): the pivot order and block
structure of Algorithms 2/3 read off R_A must equal those the recursive
oracle computes by running the algorithms (which is pinned against Theorem 2
in test_oracle_recursive.py)."""
import itertools

import numpy as np
import pytest

from oracle import oracle as o
from oracle import recursive as rc
from paper_1802_10453_gb300 import inputs
from paper_1802_10453_gb300.recursive_order import recursive_order


def _rpm_col(S, p):
    R = o.rank_profile_bruteforce(S, p)
    return [int(np.nonzero(R[i])[0][0]) if R[i].any() else -1 for i in range(S.shape[0])]


def _check(S, p):
    rec = rc.ldlt_alg2(np.array(S, dtype=object), p)
    perm, starts, rank = recursive_order(_rpm_col(S, p))
    assert perm == rec["perm"]
    assert starts == [bool(v) for v in rec["e"]]
    assert rank == rec["rank"]


@pytest.mark.parametrize("n,p", [(1, 2), (2, 2), (3, 2), (4, 2), (2, 3), (3, 3)])
def test_exhaustive_small_fields(n, p):
    pos = [(i, j) for i in range(n) for j in range(i + 1)]
    for vals in itertools.product(range(p), repeat=len(pos)):
        S = np.zeros((n, n), dtype=np.int64)
        for (i, j), v in zip(pos, vals):
            S[i, j] = S[j, i] = v
        _check(S, p)


@pytest.mark.parametrize("p", [2, 5, 65521, 2147483647])
def test_random_planted_and_uniform(p):
    rng = np.random.default_rng(p % 991)
    for t in range(30):
        n = int(rng.integers(2, 17))
        if t % 3 == 0:
            S = rng.integers(0, min(p, 1 << 30), size=(n, n)) % p
            S = np.tril(S) + np.tril(S, -1).T
        else:
            r = int(rng.integers(0, n + 1))
            A, _, _ = inputs.planted_matrix(n, r, [r // 4, r // 2][t % 2], p, 4000 + t)
            A = np.asarray(A, dtype=np.int64) % p
            S = np.tril(A) + np.tril(A, -1).T
        _check(S, p)


def test_large_order_is_fast_and_a_permutation():
    n = 16384
    rng = np.random.default_rng(1)
    idx = rng.permutation(n)
    col = [-1] * n
    for k in range(0, 6000, 2):          # 3000 pairs
        a, b = int(idx[k]), int(idx[k + 1])
        col[a], col[b] = b, a
    for k in range(6000, 9000):          # 3000 fixed points
        col[int(idx[k])] = int(idx[k])
    perm, starts, rank = recursive_order(col)
    assert sorted(perm) == list(range(n)) and rank == 9000
    assert sum(starts) == 3000
    for k in range(rank):                # blocks hold R_A's pairs and fixed points
        if starts[k]:
            assert col[perm[k]] == perm[k + 1]
        elif k == 0 or not starts[k - 1]:
            assert col[perm[k]] == perm[k]


def test_rejects_a_non_symmetric_placement():
    with pytest.raises(ValueError):
        recursive_order([1, -1])
    with pytest.raises(ValueError):
        recursive_order([5])
