"""GPU parity of ldlt_rpm_solve (A X = B from the factorisation) through the C ABI.

Every solution is compared bit for bit with the oracle's solve on the oracle's
factorisation (the two factorisations are identical: test_gpu_parity), and
checked against the defining identity A X = B mod p.  Right-hand sides outside
A's column space must be reported in the device status word.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1802_10453_gb300 as lr  # noqa: E402
from oracle import oracle as o  # noqa: E402
from paper_1802_10453_gb300 import inputs  # noqa: E402


def _gpu_solve(A, p, B, path=lr.PATH_TC):
    Ad = torch.from_numpy(np.tril(A.astype(np.int64)).astype(np.int32)).cuda()
    res = lr.factor(Ad, p, path=path)
    Bd = torch.from_numpy(np.asarray(B, dtype=np.int64).astype(np.int32)).cuda()
    X, st = lr.solve(Ad, res, Bd, check=False)
    torch.cuda.synchronize()
    return X.cpu().numpy().astype(np.int64) & 0xFFFFFFFF, int(st.item())


def _oracle_solve(A, p, B):
    f = o.ldlt_rpm(A, p)
    return o.solve_factor(f["perm"], f["L"], f["d"], f["e"], f["rank"], B, p), f["rank"]


@pytest.mark.parametrize("p", [2, 3, 65521, 8388593, 2147483647])
@pytest.mark.parametrize("n", [1, 5, 63, 64, 65, 200, 700])
def test_solve_full_rank(p, n):
    rng = np.random.default_rng(n + p % 977)
    A, _, _ = inputs.planted_matrix(n, n, n // 4, p, 300 + n)
    B = rng.integers(0, p, size=(n, 3), dtype=np.int64)
    X, st = _gpu_solve(A, p, B)
    (Xo, ok), r = _oracle_solve(A, p, B)
    assert r == n and ok and st == 0
    assert np.array_equal(X, Xo)
    assert np.array_equal(o.matmul_mod(o.symmetrize_lower(A, p), X, p), B % p)


@pytest.mark.parametrize("p", [2, 65521, 2147483647])
def test_solve_singular_consistent_and_inconsistent(p):
    rng = np.random.default_rng(p % 1013)
    n, r = 300, 190
    A, _, _ = inputs.planted_matrix(n, r, r // 4, p, 77)
    S = o.symmetrize_lower(A, p)
    B = o.matmul_mod(S, rng.integers(0, p, size=(n, 2), dtype=np.int64), p)
    X, st = _gpu_solve(A, p, B)
    (Xo, ok), rr = _oracle_solve(A, p, B)
    assert rr == r and ok and st == 0
    assert np.array_equal(X, Xo) and np.array_equal(o.matmul_mod(S, X, p), B)
    # a right-hand side outside the column space
    for trial in range(10):
        b = rng.integers(0, p, size=(n, 1), dtype=np.int64)
        if o.rank_mod_p(np.concatenate([S, b], axis=1), p) > r:
            break
    _, st = _gpu_solve(A, p, b)
    assert st == lr.LDLT_ERR_INCONSISTENT


def test_solve_after_fp64_form_and_single_vector():
    p, n = 8388593, 257
    A, _, _ = inputs.planted_matrix(n, n, 40, p, 9)
    b = np.random.default_rng(1).integers(0, p, size=n, dtype=np.int64)
    Ad = torch.from_numpy(np.tril(A.astype(np.int64)).astype(np.int32)).cuda()
    res = lr.factor(Ad, p, path=lr.PATH_FP64)
    x, _ = lr.solve(Ad, res, torch.from_numpy(b.astype(np.int32)).cuda())
    x = x.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    (Xo, ok), _ = _oracle_solve(A, p, b)
    assert ok and np.array_equal(x, Xo[:, 0])


def test_solve_n16384_planted():
    """The benchmark matrix size (rank 8192): a consistent right-hand side
    B = A y is solved and A x = B checked exactly in int64 row blocks."""
    from paper_1802_10453_gb300 import inputs_gpu
    p = 67108859
    n, r = 16384, 8192
    Ad, _ = inputs_gpu.planted_matrix(n, r, r // 4, p, inputs.SEED_BASE + 2)
    A32 = Ad.cpu().numpy()
    rng = np.random.default_rng(5)
    y = rng.integers(0, p, size=n, dtype=np.int64)

    def sym_mv(x):
        out = np.zeros(n, dtype=np.int64)
        for i0 in range(0, n, 1024):
            i1 = min(n, i0 + 1024)
            blk = A32[i0:i1, :i1].astype(np.int64) & 0xFFFFFFFF
            rows = np.arange(i0, i1)[:, None]
            cols = np.arange(i1)[None, :]
            low = np.where(cols <= rows, blk, 0)
            out[i0:i1] = (out[i0:i1] + o.matmul_mod(low, x[:i1, None], p)[:, 0]) % p
            strict = np.where(cols < rows, blk, 0)
            out[:i1] = (out[:i1] + o.matmul_mod(strict.T.copy(), x[i0:i1, None], p)[:, 0]) % p
        return out

    b = sym_mv(y)
    res = lr.factor(Ad, p)
    x, st = lr.solve(Ad, res, torch.from_numpy(b.astype(np.int32)).cuda())
    x = x.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    assert int(st.item()) == 0
    assert np.array_equal(sym_mv(x), b)
