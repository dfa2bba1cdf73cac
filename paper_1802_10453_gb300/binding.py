"""ctypes binding of libldlt_rpm.so (C ABI of include/ldlt_rpm.h).

Tensors are passed as raw device pointers and every step of the
factorisation runs in the CUDA library; the wrappers marshal arguments and
check status words.  One wrapper does host work beyond that:
factor_recursive() derives the pivot order of the recursive Algorithms 2/3
from R_A on the host (recursive_order.py, a permutation computed from the
rank profile matrix, not arithmetic of the factorisation) between two
library calls.  The library is loaded on first use and a missing library is
an error -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libldlt_rpm.so")

PATH_FP64 = 0
PATH_TC = 1
LDLT_OK = 0
LDLT_ERR_ARG = -1
LDLT_ERR_NOT_PRIME = -2
LDLT_ERR_P_RANGE = -3
LDLT_ERR_WORKSPACE = -4
LDLT_ERR_CUDA = -5
LDLT_ERR_TIMEOUT = -6
LDLT_ERR_NO_DEVICE = -7
LDLT_ERR_TOO_LARGE = -8
LDLT_ERR_INCONSISTENT = -9
LDLT_ERR_INTERNAL = -10
_NAMES = {0: "LDLT_OK", -1: "LDLT_ERR_ARG", -2: "LDLT_ERR_NOT_PRIME", -3: "LDLT_ERR_P_RANGE",
          -4: "LDLT_ERR_WORKSPACE", -5: "LDLT_ERR_CUDA", -6: "LDLT_ERR_TIMEOUT",
          -7: "LDLT_ERR_NO_DEVICE", -8: "LDLT_ERR_TOO_LARGE", -9: "LDLT_ERR_INCONSISTENT",
          -10: "LDLT_ERR_INTERNAL"}
# largest order and scratch size of ldlt_rpm_factor_noalloc (LDLT_NOALLOC_* in the header)
NOALLOC_MAX_N = 1024
NOALLOC_BYTES = 48 << 20

EXPORTS = ["ldlt_rpm_workspace_bytes", "ldlt_rpm_factor", "rpm_from_factor", "ldlt_rpm_version",
           "ldlt_rpm_set_wait_budget_ns", "ldlt_rpm_set_speculation", "ldlt_rpm_factor_noalloc",
           "ldlt_rpm_factor_batched", "ldlt_rpm_batched_workspace_bytes", "ldlt_rpm_batched_set_schedule",
           "ldlt_rpm_strict", "ldlt_rpm_solve", "ldlt_rpm_trss", "ldlt_rpm_trss_ws",
           "ldlt_rpm_trss_workspace_bytes", "ldlt_rpm_factor_given",
           "ldlt_rpm_given_workspace_bytes", "ldlt_rpm_test_drop"]
TEST_DROP_SCAN_ANSWERS = 1   # LDLT_TEST_DROP_SCAN_ANSWERS
TEST_DROP_UPDATE_COPIES = 2  # LDLT_TEST_DROP_UPDATE_COPIES
BATCH_MAX_N = 512  # LDLT_BATCH_MAX_N
SPECULATION_DEFAULT = 5  # LDLT_SPECULATION_DEFAULT


class LdltError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__("%s (%d)%s" % (_NAMES.get(code, "?"), code, (": " + what) if what else ""))
        self.code = code


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load libldlt_rpm.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError("libldlt_rpm.so is missing: run __graft_entry__.build() "
                                   "(python -m paper_1802_10453_gb300.build)")
            L = ctypes.CDLL(_LIB_PATH)
            c_i64, c_u32, c_vp, c_sz = ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t
            L.ldlt_rpm_workspace_bytes.restype = ctypes.c_int
            L.ldlt_rpm_workspace_bytes.argtypes = [c_i64, c_u32, ctypes.c_int, ctypes.POINTER(c_sz)]
            L.ldlt_rpm_factor.restype = ctypes.c_int
            L.ldlt_rpm_factor.argtypes = [c_i64, c_u32, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp,
                                          ctypes.c_int, c_vp, c_sz, c_vp]
            L.ldlt_rpm_factor_noalloc.restype = ctypes.c_int
            L.ldlt_rpm_factor_noalloc.argtypes = [c_i64, c_u32, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp,
                                                  ctypes.c_int, c_vp]
            L.ldlt_rpm_factor_given.restype = ctypes.c_int
            L.ldlt_rpm_factor_given.argtypes = [c_i64, c_u32, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp,
                                                ctypes.c_int, c_vp, c_sz, c_vp]
            L.ldlt_rpm_given_workspace_bytes.restype = ctypes.c_int
            L.ldlt_rpm_given_workspace_bytes.argtypes = [c_i64, c_u32, ctypes.c_int, ctypes.POINTER(c_sz)]
            L.ldlt_rpm_factor_batched.restype = ctypes.c_int
            L.ldlt_rpm_factor_batched.argtypes = [c_i64, c_vp, c_u32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                                  ctypes.c_int, c_vp, c_sz, c_vp]
            L.ldlt_rpm_batched_workspace_bytes.restype = ctypes.c_int
            L.ldlt_rpm_batched_workspace_bytes.argtypes = [c_i64, c_u32, ctypes.c_int, ctypes.POINTER(c_sz)]
            L.ldlt_rpm_batched_set_schedule.restype = ctypes.c_int
            L.ldlt_rpm_batched_set_schedule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.ldlt_rpm_solve.restype = ctypes.c_int
            L.ldlt_rpm_solve.argtypes = [c_i64, c_u32, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_i64, c_i64, c_vp,
                                         c_i64, c_vp, c_vp, c_sz, c_vp]
            L.ldlt_rpm_strict.restype = ctypes.c_int
            L.ldlt_rpm_strict.argtypes = [c_i64, c_u32, c_vp, c_i64, c_vp, c_vp, c_vp]
            L.ldlt_rpm_trss.restype = ctypes.c_int
            L.ldlt_rpm_trss.argtypes = [c_i64, c_u32, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp]
            L.ldlt_rpm_trss_ws.restype = ctypes.c_int
            L.ldlt_rpm_trss_ws.argtypes = [c_i64, c_u32, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_sz, c_vp]
            L.ldlt_rpm_trss_workspace_bytes.restype = ctypes.c_int
            L.ldlt_rpm_trss_workspace_bytes.argtypes = [c_i64, c_u32, ctypes.POINTER(c_sz)]
            L.rpm_from_factor.restype = ctypes.c_int
            L.rpm_from_factor.argtypes = [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]
            L.ldlt_rpm_version.restype = ctypes.c_int
            L.ldlt_rpm_version.argtypes = []
            L.ldlt_rpm_set_wait_budget_ns.restype = None
            L.ldlt_rpm_set_wait_budget_ns.argtypes = [c_i64]
            L.ldlt_rpm_set_speculation.restype = ctypes.c_int
            L.ldlt_rpm_set_speculation.argtypes = [ctypes.c_int]
            L.ldlt_rpm_test_drop.restype = ctypes.c_int
            L.ldlt_rpm_test_drop.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def workspace_bytes(n: int, p: int, path: int = PATH_TC) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().ldlt_rpm_workspace_bytes(int(n), int(p), int(path), ctypes.byref(out))
    if rc != LDLT_OK:
        raise LdltError(rc, "workspace query")
    return int(out.value)


def set_wait_budget_ns(ns: int) -> None:
    lib().ldlt_rpm_set_wait_budget_ns(int(ns))


def set_speculation(depth: int) -> None:
    rc = lib().ldlt_rpm_set_speculation(int(depth))
    if rc != LDLT_OK:
        raise LdltError(rc, "speculation depth must be in 1..16")


def test_drop(which: int) -> None:
    """Failure-detection test hook (ldlt_rpm_test_drop): drop one kind of
    internal message so that a bounded device wait runs out (0 = off)."""
    rc = lib().ldlt_rpm_test_drop(int(which))
    if rc != LDLT_OK:
        raise LdltError(rc, "test_drop: 0, TEST_DROP_SCAN_ANSWERS or TEST_DROP_UPDATE_COPIES")


def effective_ops(n: int, r: int) -> float:
    """Operation count of Section 6: r^3/3 + n^2 r - r^2 n."""
    n, r = float(n), float(r)
    return r ** 3 / 3.0 + n * n * r - r * r * n


def factor_raw(n, p, A_ptr, lda, perm_ptr, e_ptr, rank_ptr, status_ptr, path, ws_ptr, ws_bytes,
               stream_ptr) -> int:
    return lib().ldlt_rpm_factor(int(n), int(p), A_ptr, int(lda), perm_ptr, e_ptr, rank_ptr,
                                 status_ptr, int(path), ws_ptr, int(ws_bytes), stream_ptr)


_ws_cache = {}


def _workspace(nbytes: int, device):
    import torch
    key = (str(device),)
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        _ws_cache[key] = buf
    return buf


def factor(A, p: int, path: int = PATH_TC, stream=None, workspace=None, check: bool = True) -> dict:
    """Factor P^T A P = L D L^T mod p in place on the GPU.

    A: CUDA tensor of shape (n, n) and dtype int32 (residues as 32-bit words),
    rows contiguous; its lower triangle is read.  On return A holds L strictly
    below the diagonal (rows in perm order) and D on the diagonal.
    Returns dict(perm, e, rank, status) of CUDA tensors (rank, status: 1 element).
    """
    import torch
    if not A.is_cuda or A.dtype not in (torch.int32,) or A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise LdltError(LDLT_ERR_ARG, "A must be a square int32 CUDA tensor")
    if A.shape[0] > 0 and A.stride(1) != 1:
        raise LdltError(LDLT_ERR_ARG, "rows of A must be contiguous")
    n = A.shape[0]
    dev = A.device
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    e = torch.empty(n, dtype=torch.int32, device=dev)
    rank = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    nbytes = workspace_bytes(n, p, path)
    ws = workspace if workspace is not None else _workspace(nbytes, dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    lda = A.stride(0) if n > 0 else 1
    rc = factor_raw(n, p, A.data_ptr(), lda, perm.data_ptr(), e.data_ptr(), rank.data_ptr(),
                    status.data_ptr(), path, ws.data_ptr(), ws.numel(), stream.cuda_stream)
    if rc != LDLT_OK:
        raise LdltError(rc, "ldlt_rpm_factor")
    res = dict(perm=perm, e=e, rank=rank, status=status, n=n, p=p)
    if check:
        stream.synchronize()
        st = int(status.item())
        if st != 0:
            raise LdltError(st, "device status")
    return res


def given_workspace_bytes(n: int, p: int, path: int = PATH_TC) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().ldlt_rpm_given_workspace_bytes(int(n), int(p), int(path), ctypes.byref(out))
    if rc != LDLT_OK:
        raise LdltError(rc, "given workspace query")
    return int(out.value)


def factor_given(A, p: int, perm, starts, rank: int, path: int = PATH_TC, stream=None, workspace=None,
                 check: bool = True) -> dict:
    """ldlt_rpm_factor_given: L and D of P^T A P = L D L^T for a supplied pivot
    order `perm` (int sequence or int32 CUDA tensor, perm[k] = original index of
    position k), 2x2 block starts `starts` (bools, or a tensor whose non-zero
    entries mark them) and `rank`.  A (square int32 CUDA tensor, lower triangle
    read) is overwritten like factor() does.  Returns dict(perm, e, rank,
    status, n, p); with check=True raises if the device status is non-zero
    (LDLT_ERR_INCONSISTENT: the structure does not fit A)."""
    import torch
    if not A.is_cuda or A.dtype != torch.int32 or A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise LdltError(LDLT_ERR_ARG, "A must be a square int32 CUDA tensor")
    n = A.shape[0]
    if n > 0 and A.stride(1) != 1:
        raise LdltError(LDLT_ERR_ARG, "rows of A must be contiguous")
    dev = A.device
    pt = torch.as_tensor(perm, dtype=torch.int32).to(dev).contiguous().clone()
    et = (torch.as_tensor(starts).to(dev) != 0).to(torch.int32).contiguous()
    if pt.numel() != n or et.numel() != n:
        raise LdltError(LDLT_ERR_ARG, "perm and starts need n entries")
    rk = torch.tensor([int(rank)], dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    nbytes = given_workspace_bytes(n, p, path)
    ws = workspace if workspace is not None else _workspace(nbytes, dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    lda = A.stride(0) if n > 0 else 1
    rc = lib().ldlt_rpm_factor_given(n, int(p), A.data_ptr(), lda, pt.data_ptr(), et.data_ptr(), rk.data_ptr(),
                                     status.data_ptr(), int(path), ws.data_ptr(), ws.numel(), stream.cuda_stream)
    if rc != LDLT_OK:
        raise LdltError(rc, "ldlt_rpm_factor_given")
    res = dict(perm=pt, e=et, rank=rk, status=status, n=n, p=p)
    if check:
        stream.synchronize()
        st = int(status.item())
        if st != 0:
            raise LdltError(st, "device status")
    return res


def factor_recursive(A, p: int, path: int = PATH_TC, stream=None, check: bool = True) -> dict:
    """The factorisation the recursive Algorithms 2/3 compute (Section 4): their
    pivot order and block structure, with its unique L and D (odd p; p = 2 with
    in-block entry 0), in place in A like factor().

    Their order follows from R_A alone (recursive_order.py): one factor()
    pass on a copy of A gives R_A, the host derives the order, and
    factor_given() computes that factorisation.  Returns the factor_given
    result dict (perm, e, rank, status, n, p)."""
    import torch
    from .recursive_order import recursive_order
    A0 = A.clone()
    first = factor(A0, p, path=path, stream=stream, check=check)
    rpm = rpm_from_factor(first, stream=stream).cpu().tolist()
    del A0
    perm, starts, rank = recursive_order(rpm)
    return factor_given(A, p, perm, starts, rank, path=path, stream=stream, check=check)


def factor_noalloc(A, p: int, perm, e, rank, status, path: int = PATH_TC, stream=None) -> dict:
    """ldlt_rpm_factor_noalloc: factor A in place like factor(), with the
    library's own fixed scratch array instead of a workspace, for callers that
    must not allocate device memory at call time (n <= NOALLOC_MAX_N).

    The caller supplies the outputs (perm, e: int32[n]; rank: int64[1];
    status: int32[1], all on A's device); this wrapper only passes pointers and
    allocates nothing (the library call, like factor(), only enqueues: its
    first call with a given set of arguments instantiates the CUDA graph of
    the panel loop, later ones launch it again).  Calls on one device share
    the scratch array, so calls that overlap in time race; the first call on a
    device loads the module that holds the array and should come before any
    stream capture.
    Returns dict(perm, e, rank, status, n, p); read status after the stream.
    """
    import torch
    if not A.is_cuda or A.dtype != torch.int32 or A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise LdltError(LDLT_ERR_ARG, "A must be a square int32 CUDA tensor")
    n = A.shape[0]
    if n > 0 and A.stride(1) != 1:
        raise LdltError(LDLT_ERR_ARG, "rows of A must be contiguous")
    for t, dt, cnt in ((perm, torch.int32, n), (e, torch.int32, n), (rank, torch.int64, 1),
                       (status, torch.int32, 1)):
        if t.device != A.device or t.dtype != dt or t.numel() < cnt or not t.is_contiguous():
            raise LdltError(LDLT_ERR_ARG, "output tensors: perm/e int32[n], rank int64[1], status int32[1]")
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    lda = A.stride(0) if n > 0 else 1
    rc = lib().ldlt_rpm_factor_noalloc(int(n), int(p), A.data_ptr(), int(lda), perm.data_ptr(),
                                       e.data_ptr(), rank.data_ptr(), status.data_ptr(), int(path),
                                       stream.cuda_stream)
    if rc != LDLT_OK:
        raise LdltError(rc, "ldlt_rpm_factor_noalloc")
    return dict(perm=perm, e=e, rank=rank, status=status, n=n, p=p)


def batched_workspace_bytes(count: int, p: int, path: int = PATH_TC) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().ldlt_rpm_batched_workspace_bytes(int(count), int(p), int(path), ctypes.byref(out))
    if rc != LDLT_OK:
        raise LdltError(rc, "batched workspace query")
    return int(out.value)


def set_batched_schedule(kb: int, n_cut: int = 0, kb_small: int | None = None) -> None:
    rc = lib().ldlt_rpm_batched_set_schedule(int(kb), int(n_cut), int(kb if kb_small is None else kb_small))
    if rc != LDLT_OK:
        raise LdltError(rc, "batched schedule: kb in {16, 32, 64}, 0 <= n_cut <= 513, 4 <= kb_small <= kb")


class Batch:
    """Device buffers for a batch of matrices, back to back in one int32 arena.

    matrix(i) is the (n_i, n_i) view of matrix i (leading dimension n_i);
    perm(i), e(i) its outputs; rank and status hold one entry per matrix.  The
    pointer and order arrays the C ABI takes are built once here."""

    def __init__(self, ns, device="cuda"):
        import numpy as np
        import torch
        self.ns = [int(x) for x in ns]
        self.count = len(self.ns)
        dev = torch.device(device)
        sq = np.array([max(v, 0) ** 2 for v in self.ns], dtype=np.int64)
        lin = np.array([max(v, 0) for v in self.ns], dtype=np.int64)
        self._aoff = np.concatenate([[0], np.cumsum(sq)])
        self._poff = np.concatenate([[0], np.cumsum(lin)])
        self.arena = torch.zeros(max(int(self._aoff[-1]), 1), dtype=torch.int32, device=dev)
        self.perm_arena = torch.full((max(int(self._poff[-1]), 1),), -1, dtype=torch.int32, device=dev)
        self.e_arena = torch.zeros(max(int(self._poff[-1]), 1), dtype=torch.int32, device=dev)
        self.rank = torch.zeros(max(self.count, 1), dtype=torch.int64, device=dev)
        self.status = torch.zeros(max(self.count, 1), dtype=torch.int32, device=dev)

        def ptrs(t, offs):
            return torch.tensor([t.data_ptr() + 4 * int(o) for o in offs[:-1]] or [0], dtype=torch.int64,
                                device=dev)

        self.A_ptrs = ptrs(self.arena, self._aoff)
        self.perm_ptrs = ptrs(self.perm_arena, self._poff)
        self.e_ptrs = ptrs(self.e_arena, self._poff)
        self.n = torch.tensor(self.ns or [0], dtype=torch.int64, device=dev)
        self.lda = torch.tensor([max(v, 1) for v in self.ns] or [1], dtype=torch.int64, device=dev)

    def matrix(self, i):
        n = self.ns[i]
        return self.arena[int(self._aoff[i]):int(self._aoff[i + 1])].view(n, n)

    def perm(self, i):
        return self.perm_arena[int(self._poff[i]):int(self._poff[i + 1])]

    def e(self, i):
        return self.e_arena[int(self._poff[i]):int(self._poff[i + 1])]


_bws_cache = {}


def factor_batched(batch: "Batch", p: int, path: int = PATH_TC, stream=None, workspace=None,
                   check: bool = True):
    """ldlt_rpm_factor_batched over every matrix of `batch`, in place.

    Raises LdltError for a host-detected error; with check=True waits for the
    stream and raises if any matrix's status is non-zero.  Returns the status
    tensor (one int32 per matrix)."""
    import torch
    dev = batch.arena.device
    if workspace is None:
        nbytes = batched_workspace_bytes(batch.count, p, path)
        key = str(dev)
        buf = _bws_cache.get(key)
        if buf is None or buf.numel() < nbytes:
            buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
            _bws_cache[key] = buf
        workspace = buf
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    rc = lib().ldlt_rpm_factor_batched(batch.count, batch.n.data_ptr(), int(p), batch.A_ptrs.data_ptr(),
                                       batch.lda.data_ptr(), batch.perm_ptrs.data_ptr(),
                                       batch.e_ptrs.data_ptr(), batch.rank.data_ptr(),
                                       batch.status.data_ptr(), int(path), workspace.data_ptr(),
                                       workspace.numel(), stream.cuda_stream)
    if rc != LDLT_OK:
        raise LdltError(rc, "ldlt_rpm_factor_batched")
    if check:
        stream.synchronize()
        bad = (batch.status[:batch.count] != 0).nonzero()
        if bad.numel():
            i = int(bad[0, 0])
            raise LdltError(int(batch.status[i].item()), "matrix %d of the batch" % i)
    return batch.status


def solve(A, res: dict, B, stream=None, workspace=None, check: bool = True):
    """ldlt_rpm_solve: X with A_orig X = B, from the factor res = factor(A_orig)
    (A is the factored matrix in place).  B: CUDA int32 tensor (n,) or
    (n, nrhs).  Returns (X, status tensor); with check=True raises
    LdltError(LDLT_ERR_INCONSISTENT) when B is outside A's column space."""
    import torch
    n = res["n"]
    B2 = B.reshape(n, -1) if B.dim() == 1 else B
    if B2.stride(1) != 1 or B2.dtype != torch.int32 or not B2.is_cuda:
        raise LdltError(LDLT_ERR_ARG, "B must be a CUDA int32 tensor with contiguous rows")
    nrhs = B2.shape[1]
    X = torch.empty((n, nrhs), dtype=torch.int32, device=B2.device)
    status = torch.zeros(1, dtype=torch.int32, device=B2.device)
    if workspace is None:
        workspace = torch.empty(max(4 * n * nrhs, 256), dtype=torch.uint8, device=B2.device)
    if stream is None:
        stream = torch.cuda.current_stream(B2.device)
    lda = A.stride(0) if n > 0 else 1
    rc = lib().ldlt_rpm_solve(n, int(res["p"]), A.data_ptr(), lda, res["perm"].data_ptr(), res["e"].data_ptr(),
                              res["rank"].data_ptr(), B2.data_ptr(), B2.stride(0) if n else max(nrhs, 1), nrhs,
                              X.data_ptr(), max(nrhs, 1), status.data_ptr(), workspace.data_ptr(),
                              workspace.numel(), stream.cuda_stream)
    if rc != LDLT_OK:
        raise LdltError(rc, "ldlt_rpm_solve")
    if check:
        stream.synchronize()
        st = int(status.item())
        if st != 0:
            raise LdltError(st, "ldlt_rpm_solve")
    return (X.reshape(-1) if B.dim() == 1 else X), status


def strict(A, res: dict, stream=None) -> dict:
    """ldlt_rpm_strict on the output of factor() for the same A (in place):
    characteristic 2 relaxed blocks become 1x1 pivots (Section 2.2); a no-op
    for odd p.  Take the rank profile matrix (rpm_from_factor) before this."""
    import torch
    n = res["n"]
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    lda = A.stride(0) if n > 0 else 1
    rc = lib().ldlt_rpm_strict(n, int(res["p"]), A.data_ptr(), lda, res["perm"].data_ptr(), res["e"].data_ptr(),
                               stream.cuda_stream)
    if rc != LDLT_OK:
        raise LdltError(rc, "ldlt_rpm_strict")
    return res


def trss_workspace_bytes(n: int, p: int) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().ldlt_rpm_trss_workspace_bytes(int(n), int(p), ctypes.byref(out))
    if rc != LDLT_OK:
        raise LdltError(rc, "ldlt_rpm_trss_workspace_bytes")
    return int(out.value)


def trss(U, C, p: int, stream=None, check: bool = True, tensor: bool = True, workspace=None):
    """ldlt_rpm_trss_ws (tensor=True, the trailing updates on tcgen05 with a
    workspace) or ldlt_rpm_trss (CUDA-core updates), Algorithm 1: X upper
    triangular with X^T U + U^T X = C.  U and C are square CUDA int32/uint32
    tensors of the same order (U's upper triangle and C's upper triangle are
    read); C's upper triangle is overwritten by X in place; both forms give
    the same bits.  Returns the device status tensor; with check=True waits
    for the stream and raises if it is non-zero."""
    import torch
    n = int(U.shape[0])
    if tuple(U.shape) != (n, n) or tuple(C.shape) != (n, n):
        raise LdltError(LDLT_ERR_ARG, "U and C must be square of one order")
    dev = C.device
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    ldu = U.stride(0) if n > 0 else 1
    ldc = C.stride(0) if n > 0 else 1
    if tensor:
        if workspace is None:
            workspace = torch.empty(trss_workspace_bytes(n, p), dtype=torch.uint8, device=dev)
        rc = lib().ldlt_rpm_trss_ws(n, int(p), U.data_ptr(), ldu, C.data_ptr(), ldc, st.data_ptr(),
                                    workspace.data_ptr(), workspace.numel(), stream.cuda_stream)
    else:
        rc = lib().ldlt_rpm_trss(n, int(p), U.data_ptr(), ldu, C.data_ptr(), ldc, st.data_ptr(),
                                 stream.cuda_stream)
    if rc != LDLT_OK:
        raise LdltError(rc, "ldlt_rpm_trss")
    if check:
        stream.synchronize()
        code = int(st.item())
        if code != 0:
            raise LdltError(code, "ldlt_rpm_trss device status")
    return st


def rpm_from_factor(res: dict, stream=None):
    """rpm_col[i] = j where (P Psi P^T)_ij = 1, else -1 (CUDA int32 tensor)."""
    import torch
    n = res["n"]
    dev = res["perm"].device
    out = torch.empty(n, dtype=torch.int32, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    rc = lib().rpm_from_factor(n, res["perm"].data_ptr(), res["e"].data_ptr(), res["rank"].data_ptr(),
                               out.data_ptr(), stream.cuda_stream)
    if rc != LDLT_OK:
        raise LdltError(rc, "rpm_from_factor")
    return out
