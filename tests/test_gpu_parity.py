"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer work, so every comparison is bit-exact: perm, L (strictly lower part
of the returned A), D (its diagonal and e), rank and the rank profile matrix.
At sizes the oracle cannot finish quickly the factorisation is checked by
properties that pin it completely: R_A equals the planted supp(R) (Theorem 1
with lower-triangular congruence), perm is the canonical order read off R_A
(lexicographic pivoting of Algorithm 4), the block shapes of D, and
P^T A P = L D L^T on random vectors (Freivalds) -- L and D are unique once P
and the block structure are fixed.
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

PATHS = {"tc": lr.PATH_TC, "fp64": lr.PATH_FP64}


def fp64_ok(p):
    try:
        lr.workspace_bytes(4, p, lr.PATH_FP64)
        return True
    except lr.LdltError:
        return False


def gpu_factor(A_np, p, path):
    n = A_np.shape[0]
    Ad = torch.from_numpy(np.tril(np.asarray(A_np, dtype=np.int64)).astype(np.int32)).cuda()
    res = lr.factor(Ad, p, path=path)
    rpm = lr.rpm_from_factor(res)
    torch.cuda.synchronize()
    out = Ad.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    return dict(perm=res["perm"].cpu().numpy().astype(np.int64),
                Lstrict=np.tril(out, -1), d=np.diag(out).copy(),
                e=res["e"].cpu().numpy().astype(np.int64) & 0xFFFFFFFF,
                rank=int(res["rank"].item()), rpm=rpm.cpu().numpy().astype(np.int64), n=n)


def assert_parity(A_np, p, path):
    ref = o.ldlt_rpm(np.asarray(A_np, dtype=np.int64).astype(np.uint32), p)
    got = gpu_factor(A_np, p, path)
    assert got["rank"] == ref["rank"]
    assert np.array_equal(got["perm"], ref["perm"].astype(np.int64))
    assert np.array_equal(got["d"], ref["d"].astype(np.int64))
    assert np.array_equal(got["e"], ref["e"].astype(np.int64))
    assert np.array_equal(got["Lstrict"], np.tril(ref["L"].astype(np.int64), -1))
    assert np.array_equal(got["rpm"], o.rpm_from_factor(ref["perm"], ref["e"], ref["rank"]))
    return got, ref


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("p,A", [
    (7, [[0, 1], [1, 0]]), (2, [[0, 1], [1, 1]]), (7, [[0, 1], [1, 1]]),
    (5, [[0]]), (5, [[3]]), (65521, [[0, 0, 0], [0, 0, 0], [0, 0, 0]]),
])
def test_worked_examples(path, p, A):
    assert_parity(np.array(A), p, PATHS[path])


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("p", [2, 3, 257, 65521, 8388593, 67108859, 2147483647])
def test_random_small(path, p):
    if path == "fp64" and not fp64_ok(p):
        pytest.skip("p beyond the FP64 form")
    rng = np.random.default_rng(p % 1000)
    for trial in range(8):
        n = int(rng.integers(1, 40))
        kind = trial % 3
        if kind == 0:
            B = rng.integers(0, p, size=(n, n))
        else:
            B = rng.integers(0, p, size=(n, n)) * (rng.random((n, n)) < 0.2)
        A = np.tril(B) + np.tril(B, -1).T
        assert_parity(A % p, p, PATHS[path])


# sizes spanning several 64/128 tiles, ragged tails, window (256) and helper
# rows, several panels (128 pivots each)
RAGGED = [(1, 1), (31, 20), (33, 33), (65, 40), (127, 127), (129, 100), (255, 200),
          (256, 192), (257, 257), (300, 150), (513, 400), (700, 300), (1000, 1000)]


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("p", [3, 65521, 8388593, 2147483647])
@pytest.mark.parametrize("n,r", RAGGED)
def test_ragged_planted(path, p, n, r):
    if path == "fp64" and not fp64_ok(p):
        pytest.skip("p beyond the FP64 form")
    for all_pairs in (False, True):
        A, partner, _ = inputs.planted_matrix(n, r, inputs.default_pairs(r, all_pairs), p, n + r)
        got, _ = assert_parity(A, p, PATHS[path])
        assert np.array_equal(got["rpm"], partner)


@pytest.mark.parametrize("path", list(PATHS))
def test_char2(path):
    for n, r in [(40, 30), (300, 200), (600, 600)]:
        A, partner, _ = inputs.planted_matrix(n, r, r // 4, 2, 11 + n)
        got, _ = assert_parity(A, 2, PATHS[path])
        assert np.array_equal(got["rpm"], partner)


@pytest.mark.parametrize("path", list(PATHS))
def test_uniform_and_degenerate(path):
    p = 65521
    assert_parity(inputs.uniform_symmetric(700, p, 3).astype(np.int64), p, PATHS[path])
    assert_parity(np.zeros((400, 400), dtype=np.int64), p, PATHS[path])     # rank 0
    assert_parity(np.eye(300, dtype=np.int64), p, PATHS[path])              # identity
    J = np.fliplr(np.eye(300, dtype=np.int64))                              # all 2x2 pivots
    assert_parity(J, p, PATHS[path])
    A = np.zeros((500, 500), dtype=np.int64)                                # one far pair
    A[3, 480] = A[480, 3] = 5
    A[10, 10] = 1
    assert_parity(A, p, PATHS[path])


@pytest.mark.parametrize("path", list(PATHS))
def test_entries_reduced_on_ingest(path):
    p = 65521
    A, _, _ = inputs.planted_matrix(200, 150, 30, p, 5)
    big = A.astype(np.int64) + p * np.random.default_rng(1).integers(0, 3, size=A.shape)
    big = np.minimum(big, 2 ** 31 - 1)
    big = big - ((big - A) % p)  # keep big == A mod p
    ref = assert_parity(A, p, PATHS[path])[0]
    got = gpu_factor(big, p, PATHS[path])
    assert np.array_equal(got["perm"], ref["perm"]) and np.array_equal(got["Lstrict"], ref["Lstrict"])


def test_empty_matrix():
    Ad = torch.zeros((0, 0), dtype=torch.int32, device="cuda")
    res = lr.factor(Ad, 65521, path=lr.PATH_TC)
    assert int(res["rank"].item()) == 0


@pytest.mark.parametrize("path", list(PATHS))
def test_config0_planted_n256(path):
    """n = 256, r = 192, p = 65521, A = T R T^T (48 pairs + 96 fixed points)."""
    n, r, p = 256, 192, 65521
    A, partner, _ = inputs.planted_matrix(n, r, r // 4, p, inputs.SEED_BASE)
    got, ref = assert_parity(A, p, PATHS[path])
    assert got["rank"] == r and np.array_equal(got["rpm"], partner)


@pytest.mark.parametrize("path", list(PATHS))
def test_config1_uniform_n4096(path):
    """n = 4096 uniform symmetric mod 8388593, exact against the oracle."""
    from paper_1802_10453_gb300 import inputs_gpu
    n, p = 4096, 8388593
    Ad = inputs_gpu.uniform_symmetric(n, p, inputs.SEED_BASE + 1)
    A = inputs.uniform_symmetric(n, p, inputs.SEED_BASE + 1)
    assert np.array_equal(np.tril(Ad.cpu().numpy().astype(np.int64)), np.tril(A.astype(np.int64)))
    assert_parity(A, p, PATHS[path])


def _freivalds_host(A32, L32, perm, d, e, p, trials=2, seed=99, block=1024):
    """P^T A P x == L (D (L^T x)) mod p for random x, exact in int64.

    A32: the input, only its lower triangle is used; L32: the returned matrix,
    only its strict lower triangle (L) is used.  Both are processed in blocks
    of rows so that n = 32768 fits in host memory."""
    rng = np.random.default_rng(seed)
    n = A32.shape[0]

    def mulv(M, x):  # exact (M @ x) mod p for entries < 2^31, x split in 16-bit halves
        lo, hi = x & 0xFFFF, x >> 16
        return ((((M @ hi) % p) << 16) % p + (M @ lo) % p) % p

    def low_mv(M32, x, strict, transpose):
        y = np.zeros(n, dtype=np.int64)
        for i0 in range(0, n, block):
            i1 = min(n, i0 + block)
            blk = M32[i0:i1, :i1].astype(np.int64) & 0xFFFFFFFF
            rows = np.arange(i0, i1)[:, None]
            cols = np.arange(i1)[None, :]
            blk[(cols >= rows) if strict else (cols > rows)] = 0
            if transpose:
                y[:i1] = (y[:i1] + mulv(blk.T, x[i0:i1])) % p
            else:
                y[i0:i1] = mulv(blk, x[:i1])
        return y

    for _ in range(trials):
        x = rng.integers(0, p, size=n, dtype=np.int64)
        px = np.zeros(n, dtype=np.int64)
        px[perm] = x
        # S px with S symmetric from its lower part: (low + strict_low^T) px
        lhs = (low_mv(A32, px, False, False) + low_mv(A32, px, True, True)) % p
        lhs = lhs[perm]
        t = (low_mv(L32, x, True, True) + x) % p                 # L^T x (unit diagonal)
        Dt = (d * t) % p
        nxt = np.zeros(n, dtype=np.int64)
        nxt[:-1] = t[1:]
        prv = np.zeros(n, dtype=np.int64)
        prv[1:] = t[:-1] * e[:-1]
        Dt = (Dt + (e * nxt) % p + prv % p) % p
        rhs = (low_mv(L32, Dt, True, False) + Dt) % p           # L (D L^T x)
        if not np.array_equal(lhs, rhs):
            return False
    return True


def _check_planted_full_size(n, r, all_pairs, p, seed, path):
    from paper_1802_10453_gb300 import inputs_gpu
    Ad, partner = inputs_gpu.planted_matrix(n, r, inputs.default_pairs(r, all_pairs), p, seed)
    A32 = Ad.cpu().numpy()
    res = lr.factor(Ad, p, path=path)
    rpm = lr.rpm_from_factor(res).cpu().numpy().astype(np.int64)
    out32 = Ad.cpu().numpy()
    del Ad
    perm = res["perm"].cpu().numpy().astype(np.int64)
    e = res["e"].cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    rank = int(res["rank"].item())
    d = np.diag(out32).astype(np.int64) & 0xFFFFFFFF
    assert rank == r
    assert np.array_equal(rpm, partner)                       # reveals R_A = supp(R)
    perm_c, starts = o.canonical_perm_from_rpm(o.rpm_col_to_matrix(partner)) if n <= 4096 else \
        _canonical_perm_sparse(partner)
    assert np.array_equal(perm, perm_c)                       # lexicographic order
    assert np.array_equal(e != 0, starts) and np.all((d[starts] == 0))
    if p != 2:
        assert np.all(d[np.roll(starts, 1)] == 0)             # antidiagonal blocks
    assert np.all(d[r:] == 0) and np.all(e[r:] == 0)
    for i0 in range(r, n, 2048):                              # identity columns beyond r
        blk = out32[i0:i0 + 2048, r:]
        assert not np.any(np.tril(blk, i0 - r - 1))
    assert _freivalds_host(A32, out32, perm, d, e, p)


def _canonical_perm_sparse(partner):
    n = len(partner)
    perm, starts, zero = [], [], []
    placed = np.zeros(n, dtype=bool)
    for i in range(n):
        if placed[i]:
            continue
        j = partner[i]
        if j < 0:
            zero.append(i)
        elif j == i:
            perm.append(i); starts.append(False); placed[i] = True
        else:
            perm += [i, int(j)]; starts += [True, False]; placed[i] = placed[j] = True
    return np.array(perm + zero, dtype=np.int64), np.array(starts + [False] * len(zero))


@pytest.mark.parametrize("path", list(PATHS))
def test_planted_n2048_properties(path):
    n, r, p = 2048, 1500, 65521
    _check_planted_full_size(n, r, False, p, 4242, PATHS[path])


def test_config2_planted_n16384_tc():
    """n = 16384, r = 8192, p = 2^26 - 5, 2048 pairs + 4096 fixed points."""
    _check_planted_full_size(16384, 8192, False, 67108859, inputs.SEED_BASE + 2, lr.PATH_TC)


def test_config4_planted_n32768_all_pairs_tc():
    """n = 32768, r = 16384, p = 2^31 - 1, R made only of transpositions
    (8192 pairs, no fixed points): every pivot is a 2x2 antidiagonal block and
    half of the rows are zero rows found by the far scans."""
    _check_planted_full_size(32768, 16384, True, 2147483647, inputs.SEED_BASE + 4, lr.PATH_TC)


def test_planted_n28000_full_scan_fifo():
    """About 184 far rows per helper CTA: far scans answer slowly, so the
    leader's FIFO of speculative scans fills up; a scan answered with a
    partner while the FIFO is full must roll back to its own snapshot."""
    _check_planted_full_size(28000, 14000, False, 65521, 91 + 28000, lr.PATH_TC)


@pytest.mark.parametrize("depth", [1, 2, 5, 9, 16])
def test_planted_speculation_depths(depth):
    """Every speculation depth gives the same exact result.  Small depths keep
    the FIFO of speculative scans full, so rows wait for the oldest scan, are
    retaken and roll back to snapshots taken in rows where the FIFO head
    moved."""
    lr.set_speculation(depth)
    try:
        _check_planted_full_size(12000, 6000, False, 65521, 17 + depth, lr.PATH_TC)
    finally:
        lr.set_speculation(lr.SPECULATION_DEFAULT)


@pytest.mark.parametrize("n,r,pairs,p", [(1, 1, 0, 65521), (7, 5, 2, 2), (100, 60, 15, 8388593),
                                         (513, 400, 100, 2147483647), (1024, 512, 256, 67108859),
                                         (1024, 1024, 512, 65521)])
def test_gpu_planted_generator_matches_host(n, r, pairs, p):
    """The GPU generator of A = T R T^T mod p (csrc/gen_kernels.cu) gives the
    host generator's matrix (inputs.planted_matrix) element by element, and
    the same support of R."""
    from paper_1802_10453_gb300 import inputs_gpu
    seed = 4000 + n + p % 97
    Ad, partner_d = inputs_gpu.planted_matrix(n, r, pairs, p, seed)
    A, partner, _ = inputs.planted_matrix(n, r, pairs, p, seed)
    got = np.tril(Ad.cpu().numpy().astype(np.int64) & 0xFFFFFFFF)
    assert np.array_equal(got, np.tril(np.asarray(A, dtype=np.int64)))
    assert np.array_equal(np.asarray(partner_d), np.asarray(partner))


_ALL_PAIRS_REF = {}


@pytest.mark.parametrize("depth", [1, 2, 16])
def test_all_pairs_n3000_p2_31_elementwise(depth):
    """The all-pairs family of the n = 32768 workload (R made only of
    transpositions, p = 2^31 - 1) at n = 3000, element by element against the
    oracle.  Half of the rows are zero rows and every pivot is a far 2x2 pair,
    so with one or two far scans in flight the FIFO of speculative scans is
    full whenever a scan finds its partner."""
    from paper_1802_10453_gb300 import inputs_gpu
    n, r, p = 3000, 1500, 2147483647
    Ad, partner = inputs_gpu.planted_matrix(n, r, inputs.default_pairs(r, True), p, 77 + n)
    A = np.tril(Ad.cpu().numpy().astype(np.int64) & 0xFFFFFFFF)
    del Ad
    if "ref" not in _ALL_PAIRS_REF:
        _ALL_PAIRS_REF["ref"] = o.ldlt_rpm(A.astype(np.uint32), p)
    ref = _ALL_PAIRS_REF["ref"]
    lr.set_speculation(depth)
    try:
        got = gpu_factor(A, p, lr.PATH_TC)
    finally:
        lr.set_speculation(lr.SPECULATION_DEFAULT)
    assert got["rank"] == ref["rank"] == r
    assert np.array_equal(got["perm"], ref["perm"].astype(np.int64))
    assert np.array_equal(got["d"], ref["d"].astype(np.int64))
    assert np.array_equal(got["e"], ref["e"].astype(np.int64))
    assert np.array_equal(got["Lstrict"], np.tril(ref["L"].astype(np.int64), -1))
    assert np.array_equal(got["rpm"], partner)


@pytest.mark.parametrize("which,path", [("scan_answers", "tc"), ("scan_answers", "fp64"),
                                        ("update_copies", "tc")])
def test_wait_that_runs_out_reports_timeout(which, path):
    """A bounded device wait that is certain to run out is reported as
    LDLT_ERR_TIMEOUT in the status word, and the next call is bit-exact.

    The hook drops one kind of internal message: the helper CTAs never answer
    a far scan (the pivot chain's leader then waits for the oldest one), or the
    tensor-core SYRDK's copy producer stops after one stage (its MMA issuer
    then waits for a stage that never lands).  The n = 1200 planted matrix has
    600 zero rows, so its first panel issues far scans and updates 944 rows."""
    n, r, p = 1200, 600, 65521
    A, partner, _ = inputs.planted_matrix(n, r, r // 4, p, 31)
    drop = lr.TEST_DROP_SCAN_ANSWERS if which == "scan_answers" else lr.TEST_DROP_UPDATE_COPIES
    Ad = torch.from_numpy(np.tril(A).astype(np.int32)).cuda()
    lr.set_wait_budget_ns(20_000_000)
    lr.test_drop(drop)
    try:
        res = lr.factor(Ad, p, path=PATHS[path], check=False)
        torch.cuda.synchronize()
        st = int(res["status"].item())
    finally:
        lr.test_drop(0)
        lr.set_wait_budget_ns(0)
    assert st == lr.LDLT_ERR_TIMEOUT
    got, _ = assert_parity(A, p, PATHS[path])
    assert np.array_equal(got["rpm"], partner)


def test_test_drop_rejects_unknown_codes():
    with pytest.raises(lr.LdltError):
        lr.test_drop(3)
    lr.test_drop(0)


@pytest.mark.parametrize("n,kind", [(2, "worked"), (5, "uniform"), (64, "planted"), (300, "planted"),
                                    (513, "uniform"), (700, "planted")])
def test_char2_strict_transform(n, kind):
    """Section 2.2: the strict characteristic-2 form on the GPU equals the
    oracle's transform of the oracle's factorisation, bit for bit, and is a
    factorisation with 1x1 and antidiagonal blocks only."""
    p = 2
    if kind == "worked":
        A = np.array([[0, 1], [1, 1]], dtype=np.uint32)
    elif kind == "uniform":
        A = inputs.uniform_symmetric(n, p, 17 + n)
    else:
        A, _, _ = inputs.planted_matrix(n, (3 * n) // 4, n // 4, p, 19 + n)
    Ad = torch.from_numpy(np.tril(A.astype(np.int64)).astype(np.int32)).cuda()
    res = lr.factor(Ad, p)
    lr.strict(Ad, res)
    torch.cuda.synchronize()
    out = Ad.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    ref = o.ldlt_rpm(A, p)
    perm, L, d, e = o.strict_char2(ref["perm"], ref["L"], ref["d"], ref["e"])
    assert np.array_equal(res["perm"].cpu().numpy().astype(np.int64), perm)
    assert np.array_equal(np.diag(out), d)
    assert np.array_equal(res["e"].cpu().numpy().astype(np.int64) & 0xFFFFFFFF, e)
    assert np.array_equal(np.tril(out, -1), np.tril(L, -1))
    Lg = np.tril(out, -1)
    Lg[np.arange(n), np.arange(n)] = 1
    assert o.check_factor(A, perm, Lg, d, e, p)
    for k in range(n - 1):  # only 1x1 pivots and antidiagonal blocks remain
        assert e[k] == 0 or (d[k] == 0 and d[k + 1] == 0)


def test_strict_is_a_noop_for_odd_p():
    A, _, _ = inputs.planted_matrix(300, 200, 50, 65521, 23)
    Ad = torch.from_numpy(np.tril(A.astype(np.int64)).astype(np.int32)).cuda()
    res = lr.factor(Ad, 65521)
    before = (Ad.clone(), res["perm"].clone(), res["e"].clone())
    lr.strict(Ad, res)
    torch.cuda.synchronize()
    assert torch.equal(Ad, before[0]) and torch.equal(res["perm"], before[1]) and torch.equal(res["e"], before[2])


@pytest.mark.parametrize("n,pad", [(1, 3), (65, 37), (300, 1)])
def test_padded_rows_lda_above_n_leave_the_padding(n, pad):
    """A as a view of wider rows (lda = n + pad): the result is the oracle's and
    the padding (poisoned before the call) is never written."""
    p = 65521
    A, _, _ = inputs.planted_matrix(n, (3 * n) // 4, n // 8, p, 55 + n)
    poison = -559038737  # 0xDEADBEEF as int32
    buf = torch.full((n, n + pad), poison, dtype=torch.int32, device="cuda")
    Av = buf[:, :n]
    Av.copy_(torch.from_numpy(np.tril(np.asarray(A, dtype=np.int64)).astype(np.int32)))
    res = lr.factor(Av, p)
    torch.cuda.synchronize()
    ref = o.ldlt_rpm(A, p)
    out = Av.cpu().numpy().astype(np.int64)
    assert int(res["rank"].item()) == ref["rank"]
    assert np.array_equal(res["perm"].cpu().numpy(), ref["perm"])
    assert np.array_equal(np.tril(out, -1), np.tril(ref["L"].astype(np.int64), -1))
    assert np.array_equal(np.diag(out), ref["d"].astype(np.int64))
    assert bool((buf[:, n:] == poison).all())
