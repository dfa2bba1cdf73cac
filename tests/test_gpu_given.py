"""GPU parity of the given-P mode (ldlt_rpm_factor_given) through the C ABI.

The L and D of P^T A P = L D L^T are unique once the order and the blocks are
fixed (odd p; p = 2 with in-block entry 0), so:
* on Algorithm 4's structure the GPU must return the Algorithm 4 oracle's L, D
  and e bit for bit;
* on the structure of Algorithms 2/3 (the recursive oracle; a different order)
  it must return the recursive oracle's given-P result, which for odd p is the
  recursion's own L and D;
* a structure that does not fit A, or an order that is not a permutation, is
  reported in the status word."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1802_10453_gb300 as lr  # noqa: E402
from oracle import oracle as o  # noqa: E402
from oracle import recursive as rc  # noqa: E402
from paper_1802_10453_gb300 import inputs  # noqa: E402


def _lower32(A):
    return torch.from_numpy(np.tril(np.asarray(A, dtype=np.int64)).astype(np.uint32).view(np.int32)).cuda()


def _given(A, p, perm, starts, rank, check=True):
    Ad = _lower32(A)
    res = lr.factor_given(Ad, p, perm, starts, rank, check=check)
    torch.cuda.synchronize()
    M = Ad.cpu().numpy().view(np.uint32).astype(np.int64)
    return dict(L=np.tril(M, -1) + np.eye(len(M), dtype=np.int64), d=np.diag(M).copy(),
                e=res["e"].cpu().numpy().view(np.uint32).astype(np.int64),
                perm=res["perm"].cpu().numpy().astype(np.int64), rank=int(res["rank"].item()),
                status=int(res["status"].item()))


def _planted(n, p, seed, frac=0.5, pairs=0.25):
    r = int(round(n * frac))
    A, _, _ = inputs.planted_matrix(n, r, int(r * pairs), p, seed)
    return np.asarray(A, dtype=np.int64) % p


@pytest.mark.parametrize("p", [2, 3, 65521, 8388593, 2147483647])
@pytest.mark.parametrize("n", [1, 5, 64, 300, 700])
def test_given_on_algorithm4_structure_matches_oracle(p, n):
    A = _planted(n, p, 41 * n + p % 97)
    f = o.ldlt_rpm(np.tril(A).astype(np.uint32), p)
    perm = [int(v) for v in f["perm"]]
    got = _given(A, p, perm, f["e"] != 0, f["rank"])
    assert got["status"] == 0 and got["rank"] == f["rank"]
    assert np.array_equal(got["perm"], np.array(perm))
    Lo = np.tril(f["L"].astype(np.int64), -1) + np.eye(n, dtype=np.int64)
    assert np.array_equal(got["L"], Lo)
    assert np.array_equal(got["d"], f["d"].astype(np.int64))
    assert np.array_equal(got["e"], f["e"].astype(np.int64))


@pytest.mark.parametrize("p", [2, 3, 7, 65521, 2147483647])
@pytest.mark.parametrize("n", [6, 17, 40])
def test_given_on_recursive_structure_matches_oracle(p, n):
    S = np.tril(_planted(n, p, 900 + n + p % 13, frac=0.7, pairs=0.5))
    S = S + np.tril(S, -1).T
    rec = rc.ldlt_alg2(np.array(S, dtype=object), p)
    starts = [bool(v) for v in rec["e"]]
    ref = rc.factor_given_p(np.array(S, dtype=object), rec["perm"], starts, rec["rank"], p)
    got = _given(S, p, rec["perm"], starts, rec["rank"])
    assert got["status"] == 0
    assert np.array_equal(got["L"], np.array(ref["L"], dtype=np.int64))
    assert np.array_equal(got["d"], np.array(ref["d"], dtype=np.int64))
    assert np.array_equal(got["e"], np.array(ref["e"], dtype=np.int64))
    if p != 2:  # unique: the recursion's own factors
        assert np.array_equal(got["L"], np.array(rec["L"], dtype=np.int64) % p)
    R = rc.rpm_matrix(dict(perm=list(got["perm"]), e=list(got["e"]), d=list(got["d"])), n)
    assert np.array_equal(R, o.rank_profile_bruteforce(S, p))


def test_given_reports_structures_that_do_not_fit():
    p, n = 65521, 120
    A = _planted(n, p, 5)
    f = o.ldlt_rpm(np.tril(A).astype(np.uint32), p)
    perm, starts, r = [int(v) for v in f["perm"]], f["e"] != 0, f["rank"]
    # one pivot more than the rank: a zero 1x1 pivot
    assert _given(A, p, perm, starts, r + 1, check=False)["status"] == lr.LDLT_ERR_INCONSISTENT
    # a 2x2 block claimed on a 1x1 pivot with a non-zero diagonal
    k = next(i for i in range(r - 1) if not starts[i] and (i == 0 or not starts[i - 1]) and not starts[i + 1])
    bad = starts.copy()
    bad[k] = True
    assert _given(A, p, perm, bad, r, check=False)["status"] == lr.LDLT_ERR_INCONSISTENT
    # not a permutation (a repeated index, an index out of range)
    rep = list(perm)
    rep[3] = rep[4]
    assert _given(A, p, rep, starts, r, check=False)["status"] == lr.LDLT_ERR_ARG
    out = list(perm)
    out[7] = n + 5
    assert _given(A, p, out, starts, r, check=False)["status"] == lr.LDLT_ERR_ARG


def test_given_n16384_benchmark_structure():
    """The benchmark matrix refactored with its own structure: the same L, D
    (compared on sampled rows) and the planted rank profile."""
    from paper_1802_10453_gb300 import inputs_gpu
    A0, n, r, p, partner = inputs_gpu.workload_matrix("planted_n16384_r8192_p67108859")
    A1 = A0.clone()
    res = lr.factor(A1, p)
    A2 = A0.clone()
    got = lr.factor_given(A2, p, res["perm"], res["e"], int(res["rank"].item()))
    assert int(got["status"].item()) == 0
    assert torch.equal(got["e"], res["e"]) and int(got["rank"].item()) == r
    rows = torch.tensor([0, 1, 7, 4095, 8191, 8192, 12000, n - 1], device=A1.device)
    assert torch.equal(A1[rows], A2[rows])
    assert torch.equal(torch.diagonal(A1), torch.diagonal(A2))
    rpm = lr.rpm_from_factor(got).cpu().numpy()
    assert np.array_equal(rpm, partner)


@pytest.mark.parametrize("p", [2, 3, 65521, 2147483647])
@pytest.mark.parametrize("n", [7, 24, 40])
def test_factor_recursive_matches_the_recursive_oracle(p, n):
    """The recursion's order read off R_A, then the given-P mode: the GPU
    returns the factorisation Algorithms 2/3 compute (unique for odd p)."""
    S = np.tril(_planted(n, p, 77 + 3 * n + p % 7, frac=0.75, pairs=0.4))
    S = S + np.tril(S, -1).T
    rec = rc.ldlt_alg2(np.array(S, dtype=object), p)
    Ad = _lower32(S)
    res = lr.factor_recursive(Ad, p)
    M = Ad.cpu().numpy().view(np.uint32).astype(np.int64)
    L = np.tril(M, -1) + np.eye(n, dtype=np.int64)
    assert res["perm"].cpu().tolist() == rec["perm"]
    assert int(res["rank"].item()) == rec["rank"]
    assert np.array_equal(res["e"].cpu().numpy().view(np.uint32).astype(np.int64), np.array(rec["e"]))
    if p != 2:
        assert np.array_equal(L, np.array(rec["L"], dtype=np.int64) % p)
        assert np.array_equal(np.diag(M), np.array(rec["d"], dtype=np.int64))
    else:
        ref = rc.factor_given_p(np.array(S, dtype=object), rec["perm"], [bool(v) for v in rec["e"]], rec["rank"], p)
        assert np.array_equal(L, np.array(ref["L"], dtype=np.int64))
