"""GPU parity of ldlt_rpm_trss (Algorithm 1, TRSS) through the C ABI.

X (upper triangular, X^T U + U^T X = C) is unique for odd p, so the GPU's X
must equal the recursive oracle's bit for bit; for p = 2 both take x_ii = 0,
which fixes the rest.  Larger orders are checked by the defining identity
with exact host products.  Device-detected errors (a zero diagonal in U; a
characteristic-2 system with no solution) come back in the status word."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1802_10453_gb300 as lr  # noqa: E402
from oracle import oracle as o  # noqa: E402
from oracle import recursive as rc  # noqa: E402


def _inputs(n, p, seed, zero_diag_c=False):
    rng = np.random.default_rng(seed)
    hi = min(p, 1 << 31)
    U = np.triu(rng.integers(0, hi, size=(n, n), dtype=np.int64)) % p
    U[np.arange(n), np.arange(n)] = rng.integers(1, hi, size=n) % p
    for i in range(n):
        if U[i, i] == 0:
            U[i, i] = 1
    C = rng.integers(0, hi, size=(n, n), dtype=np.int64) % p
    C = np.triu(C) + np.triu(C, 1).T
    if zero_diag_c:
        C[np.arange(n), np.arange(n)] = 0
    return U, C


def _gpu(U, C, p, check=True, tensor=True):
    Ud = torch.from_numpy(U.astype(np.uint32).view(np.int32)).cuda()
    low = np.tril(C, -1) + 7  # marker values in the strict lower triangle
    Cin = np.triu(C) + np.tril(low, -1)
    Cd = torch.from_numpy(Cin.astype(np.uint32).view(np.int32)).cuda()
    st = lr.trss(Ud, Cd, p, check=check, tensor=tensor)
    torch.cuda.synchronize()
    out = Cd.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(np.tril(out, -1), np.tril(Cin, -1))  # lower triangle untouched
    return np.triu(out), int(st.item())


@pytest.mark.parametrize("p", [3, 65521, 8388593, 2147483647])
@pytest.mark.parametrize("n", [1, 2, 5, 31, 32, 33, 64, 65, 97])
def test_trss_matches_oracle(p, n):
    U, C = _inputs(n, p, n * 7 + p % 101)
    X, st = _gpu(U, C, p)
    assert st == 0
    Xo = np.array(rc.trss(U, C, p), dtype=np.int64)
    assert np.array_equal(X, Xo)


@pytest.mark.parametrize("n", [1, 33, 70])
def test_trss_characteristic_2(n):
    U, C = _inputs(n, 2, 11 + n, zero_diag_c=True)
    # a consistent right-hand side: C = Y^T U + U^T Y for an upper Y
    Y = np.triu(np.random.default_rng(n).integers(0, 2, size=(n, n)))
    C = (Y.T @ U + U.T @ Y) % 2
    X, st = _gpu(U, C, 2)
    assert st == 0
    assert np.array_equal(X, np.array(rc.trss(U, C, 2), dtype=np.int64))
    assert np.array_equal((X.T @ U + U.T @ X) % 2, C)
    if n > 1:
        C2 = C.copy()
        C2[n - 1, n - 1] = 1  # the diagonal of X^T U + U^T X is zero mod 2
        _, st = _gpu(U, C2, 2, check=False)
        assert st == lr.LDLT_ERR_INCONSISTENT


@pytest.mark.parametrize("n,p", [(300, 65521), (1000, 8388593), (700, 2147483647)])
def test_trss_identity_larger(n, p):
    U, C = _inputs(n, p, n + 3)
    X, st = _gpu(U, C, p)
    assert st == 0
    assert not np.any(np.tril(X, -1))
    lhs = (o.matmul_mod(X.T, U, p) + o.matmul_mod(U.T, X, p)) % p
    assert np.array_equal(lhs, C)


@pytest.mark.parametrize("n,p", [(257, 3), (600, 65521), (300, 2), (513, 8388593), (1000, 2147483647),
                                 (700, 67108859)])
def test_trss_tensor_update_equals_cuda_core(n, p):
    """The tcgen05 trailing update (orders >= 256: tile tails, several block
    steps on tensor cores, the last ones on CUDA cores) gives the same X bit
    for bit as the CUDA-core form, which the oracle pins at small orders; for
    odd p the identity X^T U + U^T X = C holds exactly."""
    if p == 2:
        U, _ = _inputs(n, 2, 9 + n)
        Y = np.triu(np.random.default_rng(n).integers(0, 2, size=(n, n)))
        C = (o.matmul_mod(Y.T, U, 2) + o.matmul_mod(U.T, Y, 2)) % 2
    else:
        U, C = _inputs(n, p, 31 * n + p % 97)
    Xt, st = _gpu(U, C, p, tensor=True)
    Xc, sc = _gpu(U, C, p, tensor=False)
    assert st == sc == 0
    assert np.array_equal(Xt, Xc)
    assert np.array_equal((o.matmul_mod(Xt.T, U, p) + o.matmul_mod(U.T, Xt, p)) % p, C)


def test_trss_reports_zero_diagonal_and_bad_arguments():
    U, C = _inputs(40, 65521, 5)
    U[17, 17] = 0
    _, st = _gpu(U, C, 65521, check=False)
    assert st == lr.LDLT_ERR_ARG
    with pytest.raises(lr.LdltError):
        lr.trss(torch.zeros((3, 3), dtype=torch.int32, device="cuda"),
                torch.zeros((3, 3), dtype=torch.int32, device="cuda"), 65520)  # composite p
    _, st = _gpu(np.zeros((0, 0), dtype=np.int64), np.zeros((0, 0), dtype=np.int64), 7)
    assert st == 0
