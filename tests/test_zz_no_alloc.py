"""ldlt_rpm_factor_noalloc: the factorisation for callers that cannot allocate.

A caller that has handed all of its device memory to its own pool, or that
runs a loop where a cudaMalloc (which may synchronise the device) is not
acceptable, calls this entry point: it takes no workspace and keeps its
scratch in one fixed array inside the library (at most LDLT_NOALLOC_MAX_N
rows).  These tests call it through the C ABI, twice in a row with different
problems so that anything the first call left in the shared array would show
up in the second, and require the outputs to equal those of ldlt_rpm_factor
bit for bit.  The file is named so that pytest collects it last: it must pass
both in a fresh process and after every other test has run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1802_10453_gb300 as lr  # noqa: E402
from paper_1802_10453_gb300 import inputs  # noqa: E402


def _tensors(A_np):
    n = A_np.shape[0]
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(np.tril(A_np.astype(np.int64)).astype(np.int32)).to(dev)
    return dict(A=A, perm=torch.full((n,), -7, dtype=torch.int32, device=dev),
                e=torch.full((n,), -7, dtype=torch.int32, device=dev),
                rank=torch.full((1,), -7, dtype=torch.int64, device=dev),
                status=torch.full((1,), -7, dtype=torch.int32, device=dev))


def _noalloc_raw(t, p, path):
    """One call of the new entry point through the C ABI (ctypes), default stream."""
    A = t["A"]
    n = A.shape[0]
    return lr.lib().ldlt_rpm_factor_noalloc(n, p, A.data_ptr(), max(n, 1), t["perm"].data_ptr(),
                                            t["e"].data_ptr(), t["rank"].data_ptr(),
                                            t["status"].data_ptr(), path, None)


def _host(t):
    return {k: v.cpu().numpy() for k, v in t.items()}


def _with_workspace(A_np, p, path, workspace=None):
    t = _tensors(A_np)
    res = lr.factor(t["A"], p, path=path, workspace=workspace)
    torch.cuda.synchronize()
    return _host(dict(A=t["A"], perm=res["perm"], e=res["e"], rank=res["rank"], status=res["status"]))


def _same(got, ref):
    n = ref["A"].shape[0]
    assert int(got["status"][0]) == 0
    assert int(got["rank"][0]) == int(ref["rank"][0])
    assert np.array_equal(got["perm"], ref["perm"])
    assert np.array_equal(got["e"], ref["e"])
    # L strictly below the diagonal and D on it; the upper triangle is unspecified
    assert np.array_equal(np.tril(got["A"]), np.tril(ref["A"]))
    assert n == got["A"].shape[0]


# Two problems per sequence, run back to back on the shared array: the first at
# the maximum order, the second smaller, with another prime and rank, so that
# stale rows, pivots or event records of the first call would corrupt it.
SEQUENCES = {
    "tc_then_tc": [(1024, 700, 2147483647, lr.PATH_TC), (517, 517, 65521, lr.PATH_TC)],
    "tc_then_fp64": [(900, 450, 8388593, lr.PATH_TC), (640, 300, 65521, lr.PATH_FP64)],
    "char2_then_odd": [(800, 500, 2, lr.PATH_TC), (300, 150, 3, lr.PATH_TC)],
}


@pytest.mark.parametrize("name", sorted(SEQUENCES))
def test_two_calls_in_a_row_match_workspace_entry(name):
    probs = []
    for i, (n, r, p, path) in enumerate(SEQUENCES[name]):
        A, _, _ = inputs.planted_matrix(n, r, inputs.default_pairs(r), p, 1000 + 17 * i + n)
        probs.append((A, p, path, _with_workspace(A, p, path)))
    got = []
    for A, p, path, _ in probs:
        t = _tensors(A)
        assert _noalloc_raw(t, p, path) == lr.LDLT_OK
        torch.cuda.synchronize()
        got.append(_host(t))
    for (A, p, path, ref), g in zip(probs, got):
        _same(g, ref)


def test_second_call_takes_no_device_memory():
    A, _, _ = inputs.planted_matrix(600, 400, inputs.default_pairs(400), 65521, 4242)
    ref = _with_workspace(A, 65521, lr.PATH_TC)
    t1, t2 = _tensors(A), _tensors(A)
    assert _noalloc_raw(t1, 65521, lr.PATH_TC) == lr.LDLT_OK  # may load the module holding the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    assert _noalloc_raw(t2, 65521, lr.PATH_TC) == lr.LDLT_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    _same(_host(t1), ref)
    _same(_host(t2), ref)


def test_dirty_scratch_is_harmless():
    """The shared array is never cleared between calls: the factorisation
    clears what must start at zero itself.  The same holds for a caller's
    workspace filled with 0xFF bytes, which is the evidence checked here
    against a call of the no-allocation entry point."""
    A, _, _ = inputs.planted_matrix(700, 520, inputs.default_pairs(520), 67108859, 99)
    nbytes = lr.workspace_bytes(700, 67108859, lr.PATH_TC)
    ws = torch.full((nbytes,), 0xFF, dtype=torch.uint8, device="cuda")
    ref = _with_workspace(A, 67108859, lr.PATH_TC, workspace=ws)
    t = _tensors(A)
    assert _noalloc_raw(t, 67108859, lr.PATH_TC) == lr.LDLT_OK
    torch.cuda.synchronize()
    _same(_host(t), ref)


def test_binding_and_limits():
    # the Python wrapper passes the caller's outputs through unchanged
    A, _, _ = inputs.planted_matrix(300, 200, 40, 65521, 7)
    ref = _with_workspace(A, 65521, lr.PATH_FP64)
    t = _tensors(A)
    res = lr.factor_noalloc(t["A"], 65521, t["perm"], t["e"], t["rank"], t["status"], path=lr.PATH_FP64)
    torch.cuda.synchronize()
    assert res["perm"].data_ptr() == t["perm"].data_ptr()
    _same(_host(t), ref)
    # n = 0: rank 0, nothing else touched
    t0 = _tensors(np.zeros((0, 0), dtype=np.uint32))
    assert _noalloc_raw(t0, 65521, lr.PATH_TC) == lr.LDLT_OK
    torch.cuda.synchronize()
    assert int(t0["rank"][0]) == 0 and int(t0["status"][0]) == 0
    # one row above the maximum is refused on the host, before any device work
    big = lr.NOALLOC_MAX_N + 1
    rc = lr.lib().ldlt_rpm_factor_noalloc(big, 65521, ctypes.c_void_p(16), big, ctypes.c_void_p(16),
                                          ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                          lr.PATH_TC, None)
    assert rc == lr.LDLT_ERR_TOO_LARGE
    with pytest.raises(lr.LdltError):
        Abig = torch.zeros((big, big), dtype=torch.int32, device="cuda")
        tb = _tensors(np.zeros((1, 1), dtype=np.uint32))
        pb = torch.zeros(big, dtype=torch.int32, device="cuda")
        lr.factor_noalloc(Abig, 65521, pb, pb.clone(), tb["rank"], tb["status"])
