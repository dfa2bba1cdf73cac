"""GPU parity of the batched schedule (ldlt_rpm_factor_batched) through the C ABI.

Every matrix of a batch must come out exactly as the CPU oracle factors it
alone (perm, L, D, e, rank: integer work, bit-exact), whatever its order,
rank, prime or position in the queue, and whatever panel width and cutoff the
schedule uses.  At the full batch size (4096 matrices, n in [32, 512]) every
matrix is checked by properties that pin P completely (rank = planted rank,
perm = the canonical order read off the planted R_A), and a sample against the
oracle and against the single-matrix entry point.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1802_10453_gb300 as lr  # noqa: E402
from oracle import oracle as o  # noqa: E402
from paper_1802_10453_gb300 import inputs, inputs_gpu  # noqa: E402


def _fill_host(batch, mats):
    for i, A in enumerate(mats):
        if A.shape[0]:
            batch.matrix(i).copy_(torch.from_numpy(np.tril(A.astype(np.int64)).astype(np.int32)))


def _out(batch, i):
    n = batch.ns[i]
    M = batch.matrix(i).cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    return dict(perm=batch.perm(i).cpu().numpy().astype(np.int64),
                Lstrict=np.tril(M, -1), d=np.diag(M).copy(),
                e=batch.e(i).cpu().numpy().astype(np.int64) & 0xFFFFFFFF,
                rank=int(batch.rank[i].item()), status=int(batch.status[i].item()), n=n)


def _assert_oracle(A, p, got):
    ref = o.ldlt_rpm(np.asarray(A, dtype=np.int64).astype(np.uint32), p)
    assert got["status"] == 0
    assert got["rank"] == ref["rank"]
    assert np.array_equal(got["perm"], ref["perm"].astype(np.int64))
    assert np.array_equal(got["d"], ref["d"].astype(np.int64))
    assert np.array_equal(got["e"], ref["e"].astype(np.int64))
    assert np.array_equal(got["Lstrict"], np.tril(ref["L"].astype(np.int64), -1))


EDGE_N = [1, 2, 3, 4, 5, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 300, 511, 512]


def _mixed_batch(p, seed, extra=24):
    rng = np.random.default_rng(seed)
    ns = EDGE_N + [int(x) for x in rng.integers(1, 513, size=extra)]
    mats = []
    for i, n in enumerate(ns):
        kind = i % 4
        if kind == 3:
            A = inputs.uniform_symmetric(n, p, seed + i)
        else:
            r = [n, (3 * n) // 4, n // 4][kind]
            A, _, _ = inputs.planted_matrix(n, r, r // 4 if kind != 1 else r // 2, p, seed + i)
        mats.append(A)
    return ns, mats


@pytest.mark.parametrize("p", [65521, 2, 3, 8388593, 2147483647])
def test_batched_matches_oracle(p):
    ns, mats = _mixed_batch(p, 700 + (p % 97))
    batch = lr.Batch(ns)
    _fill_host(batch, mats)
    lr.factor_batched(batch, p)
    for i, A in enumerate(mats):
        _assert_oracle(A, p, _out(batch, i))


@pytest.mark.parametrize("kb,n_cut,kb_small", [(16, 0, 16), (64, 0, 64), (64, 200, 8), (32, 513, 4)])
def test_schedule_does_not_change_results(kb, n_cut, kb_small):
    p = 65521
    ns, mats = _mixed_batch(p, 911, extra=8)
    batch = lr.Batch(ns)
    _fill_host(batch, mats)
    try:
        lr.set_batched_schedule(kb, n_cut, kb_small)
        lr.factor_batched(batch, p)
    finally:
        lr.set_batched_schedule(32, 0, 32)
    for i, A in enumerate(mats):
        _assert_oracle(A, p, _out(batch, i))


def test_invalid_entries_are_reported_per_matrix():
    p = 65521
    ns = [40, 0, 70]
    A0, _, _ = inputs.planted_matrix(40, 30, 7, p, 5)
    A2, _, _ = inputs.planted_matrix(70, 50, 12, p, 6)
    batch = lr.Batch(ns)
    _fill_host(batch, [A0, np.zeros((0, 0), np.uint32), A2])
    # second matrix: order above the batched maximum; third: lda below n
    batch.n[1] = lr.BATCH_MAX_N + 1
    batch.lda[2] = 69
    lr.factor_batched(batch, p, check=False)
    torch.cuda.synchronize()
    st = batch.status.cpu().numpy()
    assert st[0] == 0 and st[1] == lr.LDLT_ERR_ARG and st[2] == lr.LDLT_ERR_ARG
    _assert_oracle(A0, p, _out(batch, 0))
    # an empty matrix is fine
    b0 = lr.Batch([0, 3])
    _fill_host(b0, [np.zeros((0, 0), np.uint32), np.array([[0, 0, 0], [1, 0, 0], [0, 0, 5]], np.uint32)])
    lr.factor_batched(b0, 7)
    assert int(b0.rank[0].item()) == 0
    _assert_oracle(np.array([[0, 1, 0], [1, 0, 0], [0, 0, 5]]), 7, _out(b0, 1))


def test_small_workspace_runs_fewer_ctas():
    p = 65521
    ns, mats = _mixed_batch(p, 1234, extra=4)
    batch = lr.Batch(ns)
    _fill_host(batch, mats)
    header = lr.batched_workspace_bytes(len(ns), p) - min(len(ns), 640) * (1 << 20)
    ws = torch.empty(header + 3 * (1 << 20), dtype=torch.uint8, device="cuda")  # three CTAs
    lr.factor_batched(batch, p, workspace=ws)
    for i, A in enumerate(mats):
        _assert_oracle(A, p, _out(batch, i))


def _canonical_perm(partner):
    n = len(partner)
    perm, zero = [], []
    placed = np.zeros(n, dtype=bool)
    for i in range(n):
        if placed[i]:
            continue
        j = partner[i]
        if j < 0:
            zero.append(i)
        elif j == i:
            perm.append(i)
            placed[i] = True
        else:
            perm += [i, int(j)]
            placed[i] = placed[j] = True
    return np.array(perm + zero, dtype=np.int64)


def test_config3_batch4096_planted():
    """4096 matrices, n uniform in [32, 512], r uniform in [n/4, n], p = 65521."""
    count, n_lo, n_hi, p = inputs.BATCH_WORKLOADS["batch4096_n32to512_p65521"]
    seed = inputs.SEED_BASE + 3
    ns, rs = inputs.batch_shapes(count, n_lo, n_hi, seed)
    batch = lr.Batch(ns)
    partners = inputs_gpu.planted_batch(batch, rs, p, seed)
    rng = np.random.default_rng(3)
    sample = sorted(set(int(x) for x in rng.choice(count, size=24, replace=False)) | {int(np.argmax(ns))})
    inputs_host = {i: batch.matrix(i).cpu().numpy().astype(np.int64) for i in sample}
    lr.factor_batched(batch, p)
    ranks = batch.rank[:count].cpu().numpy()
    assert np.array_equal(ranks, rs)
    pa = batch.perm_arena.cpu().numpy().astype(np.int64)
    off = 0
    for i in range(count):
        n = int(ns[i])
        assert np.array_equal(pa[off:off + n], _canonical_perm(partners[i])), i
        off += n
    for i in sample:
        Alow = inputs_host[i]
        got = _out(batch, i)
        _assert_oracle(Alow + np.tril(Alow, -1).T, p, got)
        # the single-matrix entry point gives the same bits
        Ad = torch.from_numpy(Alow.astype(np.int32)).cuda()
        res = lr.factor(Ad, p)
        M = Ad.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
        assert np.array_equal(np.tril(M, -1), got["Lstrict"]) and np.array_equal(np.diag(M), got["d"])
        assert np.array_equal(res["perm"].cpu().numpy(), got["perm"])


def test_upper_triangle_untouched():
    p = 65521
    ns, mats = _mixed_batch(p, 4321, extra=4)
    batch = lr.Batch(ns)
    for i, A in enumerate(mats):
        n = A.shape[0]
        full = np.tril(A.astype(np.int64)) + np.triu(np.full((n, n), 0x5A5A5A5, dtype=np.int64), 1)
        batch.matrix(i).copy_(torch.from_numpy(full.astype(np.int32)))
    lr.factor_batched(batch, p)
    for i, A in enumerate(mats):
        n = A.shape[0]
        M = batch.matrix(i).cpu().numpy().astype(np.int64)
        assert np.all(np.triu(M, 1) == np.triu(np.full((n, n), 0x5A5A5A5, dtype=np.int64), 1))
        _assert_oracle(A, p, _out(batch, i))


def test_batched_call_replays_from_a_cuda_graph():
    """The batched call enqueues a memset and two kernels and reads nothing
    back, so it can be captured once and replayed."""
    p = 65521
    ns, mats = _mixed_batch(p, 2468, extra=6)
    batch = lr.Batch(ns)
    _fill_host(batch, mats)
    src = batch.arena.clone()
    ws = torch.empty(lr.batched_workspace_bytes(len(ns), p), dtype=torch.uint8, device="cuda")
    lr.factor_batched(batch, p, workspace=ws)  # warm-up outside the capture
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lr.factor_batched(batch, p, workspace=ws, stream=torch.cuda.current_stream(), check=False)
    for _ in range(2):
        batch.arena.copy_(src)
        batch.rank.zero_()
        g.replay()
        torch.cuda.synchronize()
        for i, A in enumerate(mats):
            _assert_oracle(A, p, _out(batch, i))


def test_autotuner_keeps_results_and_inputs():
    p = 65521
    ns, mats = _mixed_batch(p, 1357, extra=8)
    batch = lr.Batch(ns)
    _fill_host(batch, mats)
    before = batch.arena.clone()
    try:
        res = lr.tune_batched(batch, p, candidates=((32, 0, 32), (16, 0, 16), (32, 300, 8)), reps=1)
        assert res["best"] in res["ms"] and all(v > 0 for v in res["ms"].values())
        assert torch.equal(batch.arena, before)      # the inputs are back in place
        lr.factor_batched(batch, p)                  # with the chosen schedule
    finally:
        lr.set_batched_schedule(32, 0, 32)
    for i, A in enumerate(mats):
        _assert_oracle(A, p, _out(batch, i))


def test_online_tuner_over_a_stream_matches_the_oracle():
    """A stream of batches through OnlineTuner: every candidate is tried on a
    real batch, times are taken in, and every matrix of every batch is exactly
    the oracle's, whichever schedule ran it."""
    p = 65521
    cands = ((32, 0, 32), (16, 0, 16), (32, 200, 16))
    tuner = lr.OnlineTuner(p, candidates=cands, explore_every=3)
    try:
        for j in range(7):
            ns, mats = _mixed_batch(p, 4242 + j, extra=4)
            batch = lr.Batch(ns)
            _fill_host(batch, mats)
            tuner.factor(batch)
            torch.cuda.synchronize()
            for i in range(0, len(mats), 3):
                _assert_oracle(mats[i], p, _out(batch, i))
            assert int((batch.status != 0).sum().item()) == 0
        tuner.flush()
    finally:
        lr.set_batched_schedule(32, 0, 32)
    assert [c for _, c in tuner.history[:3]] == list(cands)
    assert set(tuner.cost) == set(cands) and all(v > 0 for v in tuner.cost.values())
    assert tuner.best in cands
