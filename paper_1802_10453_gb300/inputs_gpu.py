"""GPU side of the seeded generator (libldlt_gen.so), same definitions as inputs.py.

The support of R (O(n) data) is drawn on the host by ``inputs.planted_support``;
the O(n^2 r) product T R T^T runs on the GPU.  Only the lower triangle of the
returned matrix is filled (the factorisation reads nothing else).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libldlt_gen.so")
_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError("libldlt_gen.so is missing: run __graft_entry__.build()")
            L = ctypes.CDLL(_LIB_PATH)
            c_i64, c_u32, c_u64, c_vp = ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
            L.ldlt_gen_planted_ws_bytes.restype = ctypes.c_size_t
            L.ldlt_gen_planted_ws_bytes.argtypes = [c_i64, ctypes.c_int]
            L.ldlt_gen_planted.restype = ctypes.c_int
            L.ldlt_gen_planted.argtypes = [c_i64, c_u32, c_u64, ctypes.c_int, c_vp, c_vp, c_vp, c_vp,
                                           c_i64, c_vp, c_vp]
            L.ldlt_gen_uniform.restype = ctypes.c_int
            L.ldlt_gen_uniform.argtypes = [c_i64, c_u32, c_u64, c_vp, c_i64, c_vp]
            _lib = L
    return _lib


def planted_terms(partner, scale):
    """(k_q, p_q, s_q): one term per support index, R[k, p] = s."""
    sup = np.nonzero(np.asarray(partner) >= 0)[0]
    kq = sup.astype(np.int32)
    pq = np.asarray(partner)[sup].astype(np.int32)
    sq = np.asarray(scale)[sup].astype(np.uint32)
    return kq, pq, sq


def planted_matrix(n, r, npairs, p, seed, device="cuda", out=None):
    """A = T R T^T mod p on the GPU.  Returns (A int32 CUDA tensor, partner)."""
    import torch
    partner, scale = inputs.planted_support(n, r, npairs, p, seed)
    kq, pq, sq = planted_terms(partner, scale)
    A = out if out is not None else torch.zeros((n, n), dtype=torch.int32, device=device)
    L = _load()
    nterms = len(kq)
    kq_t = torch.from_numpy(kq).to(device)
    pq_t = torch.from_numpy(pq).to(device)
    sq_t = torch.from_numpy(sq.view(np.int32)).to(device)
    ws = torch.empty(int(L.ldlt_gen_planted_ws_bytes(n, nterms)), dtype=torch.uint8, device=device)
    keyT = inputs.derive_key(seed, inputs.TAG_T)
    st = torch.cuda.current_stream(A.device).cuda_stream
    rc = L.ldlt_gen_planted(n, p, keyT, nterms, kq_t.data_ptr(), pq_t.data_ptr(), sq_t.data_ptr(),
                            A.data_ptr(), A.stride(0), ws.data_ptr(), st)
    if rc != 0:
        raise RuntimeError("ldlt_gen_planted failed: %d" % rc)
    torch.cuda.current_stream(A.device).synchronize()
    del ws
    return A, partner


def planted_batch(batch, rs, p, seed, all_pairs=False):
    """Fill every matrix of a binding.Batch with its planted matrix: matrix i
    has order batch.ns[i], rank rs[i], default_pairs(rs[i]) pairs and seed
    inputs.batch_seed(seed, i).  Returns the list of partner arrays."""
    import torch
    L = _load()
    dev = batch.arena.device
    st = torch.cuda.current_stream(dev)
    nmax = max(batch.ns) if batch.ns else 0
    ws = torch.empty(max(int(L.ldlt_gen_planted_ws_bytes(nmax, nmax)), 256), dtype=torch.uint8, device=dev)
    keep, partners = [], []
    for i, n in enumerate(batch.ns):
        r = int(rs[i])
        s_i = inputs.batch_seed(seed, i)
        partner, scale = inputs.planted_support(n, r, inputs.default_pairs(r, all_pairs), p, s_i)
        kq, pq, sq = planted_terms(partner, scale)
        kq_t = torch.from_numpy(kq).to(dev, non_blocking=False)
        pq_t = torch.from_numpy(pq).to(dev)
        sq_t = torch.from_numpy(sq.view(np.int32)).to(dev)
        keep.append((kq_t, pq_t, sq_t))
        A = batch.matrix(i)
        rc = L.ldlt_gen_planted(n, p, inputs.derive_key(s_i, inputs.TAG_T), len(kq), kq_t.data_ptr(),
                                pq_t.data_ptr(), sq_t.data_ptr(), A.data_ptr(), max(n, 1), ws.data_ptr(),
                                st.cuda_stream)
        if rc != 0:
            raise RuntimeError("ldlt_gen_planted failed: %d" % rc)
        partners.append(partner)
    st.synchronize()
    del keep, ws
    return partners


def uniform_symmetric(n, p, seed, device="cuda", out=None):
    import torch
    A = out if out is not None else torch.zeros((n, n), dtype=torch.int32, device=device)
    keyU = inputs.derive_key(seed, inputs.TAG_UNIFORM)
    rc = _load().ldlt_gen_uniform(n, p, keyU, A.data_ptr(), A.stride(0),
                                  torch.cuda.current_stream(A.device).cuda_stream)
    if rc != 0:
        raise RuntimeError("ldlt_gen_uniform failed: %d" % rc)
    return A


def workload_matrix(name, device="cuda"):
    """The named workload of inputs.WORKLOADS on the GPU: (A, n, r_planted, p, partner or None)."""
    kind, n, r, p, all_pairs = inputs.WORKLOADS[name]
    seed = inputs.SEED_BASE + list(inputs.WORKLOADS).index(name)
    if kind == "planted":
        A, partner = planted_matrix(n, r, inputs.default_pairs(r, all_pairs), p, seed, device)
        return A, n, r, p, partner
    return uniform_symmetric(n, p, seed, device), n, None, p, None
