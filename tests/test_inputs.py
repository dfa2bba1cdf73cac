"""The seeded generator: structure, determinism, published SplitMix64 values."""
import numpy as np

from paper_1802_10453_gb300 import inputs


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: the first outputs of the published generator
    # (state += 0x9E3779B97F4A7C15; return mix(state)).
    assert int(inputs.stream(0, [0])[0]) == 0xE220A8397B1DCDAF
    assert int(inputs.stream(0, [1])[0]) == 0x6E789E6AA1B965F4
    assert int(inputs.stream(0, [2])[0]) == 0x06C45D188009454F


def test_T_unit_lower():
    T = inputs.T_matrix(20, 65521, 3)
    assert np.array_equal(np.diag(T), np.ones(20))
    assert not np.triu(T, 1).any()
    assert (T >= 0).all() and (T < 65521).all()


def test_planted_support_shape():
    for n, r, pairs in [(50, 30, 7), (64, 64, 32), (40, 0, 0), (33, 20, 10)]:
        partner, scale = inputs.planted_support(n, r, pairs, 101, 9)
        sup = np.nonzero(partner >= 0)[0]
        assert len(sup) == r
        fixed = [i for i in sup if partner[i] == i]
        assert len(fixed) == r - 2 * pairs
        for i in sup:
            assert partner[partner[i]] == i
            assert 1 <= scale[i] < 101
            assert scale[partner[i]] == scale[i]


def test_planted_matrix_symmetric_and_deterministic():
    A1, p1, s1 = inputs.planted_matrix(30, 20, 5, 65521, 4)
    A2, p2, s2 = inputs.planted_matrix(30, 20, 5, 65521, 4)
    assert np.array_equal(A1, A2) and np.array_equal(p1, p2)
    assert np.array_equal(A1, A1.T)
    A3, _, _ = inputs.planted_matrix(30, 20, 5, 65521, 5)
    assert not np.array_equal(A1, A3)


def test_uniform_symmetric():
    A = inputs.uniform_symmetric(17, 8388593, 2)
    assert np.array_equal(A, A.T)
    assert A.max() < 8388593
