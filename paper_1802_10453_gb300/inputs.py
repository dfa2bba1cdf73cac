"""Seeded synthetic inputs for the symmetric rank-profile factorisation.

This module holds no arithmetic of the factorisation itself; it only draws
matrices.  Both the CUDA path (tests, bench) and the CPU oracle take their
inputs from here, so the two sides see the same bits.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
the k-th output of the stream keyed by ``key`` is ``mix64(key + (k+1)*gamma)``
with gamma = 0x9E3779B97F4A7C15 and mix64 the SplitMix64 finaliser.  A value
in [0, p) is ``((out >> 32) * p) >> 32``.  The GPU generator in
``csrc/gen_kernels.cu`` implements the same definition and is checked against
this one.

Workloads (the matrix families of the paper's Section 6 experiments):
* planted rank profile:  A = T R T^T mod p, T unit lower triangular with
  uniform entries below the diagonal, R a symmetric partial permutation with
  non-zero scalings.  Lower-triangular congruence keeps every leading block's
  rank, so the rank profile matrix of A is supp(R).
* uniform symmetric: entries i.i.d. uniform in [0, p) mirrored (generic rank
  profile with high probability).
* batch: many independent planted matrices of uneven order n_i and rank r_i
  (orders below the recursion threshold of Section 6).
"""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
KEYMUL = 0xD1B54A32D192ED03

TAG_T = 1      # entries of T
TAG_SUPPORT = 2  # choice and pairing of the support of R
TAG_SCALE = 3  # scalings of R
TAG_UNIFORM = 4  # uniform symmetric matrix
TAG_BATCH = 5  # orders and ranks of the matrices of a batch


def mix64_scalar(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * MIX1) & M64
    z = ((z ^ (z >> 27)) * MIX2) & M64
    return z ^ (z >> 31)


def derive_key(seed: int, tag: int) -> int:
    return mix64_scalar((seed + tag * KEYMUL) & M64)


def _mix64(z):
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def stream(key: int, ctr):
    """SplitMix64 outputs number ``ctr`` (array) of the stream ``key``."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (ctr + np.uint64(1)) * np.uint64(GAMMA)
    return _mix64(z)


def uniform_mod(key: int, ctr, p: int):
    """Values in [0, p): ((out >> 32) * p) >> 32."""
    hi = stream(key, ctr) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return ((hi * np.uint64(p)) >> np.uint64(32)).astype(np.int64)


def T_matrix(n: int, p: int, seed: int):
    """Unit lower triangular T: T[i, j] = uniform(key_T, i*n + j) for j < i."""
    key = derive_key(seed, TAG_T)
    i, j = np.meshgrid(np.arange(n, dtype=np.uint64), np.arange(n, dtype=np.uint64), indexing="ij")
    vals = uniform_mod(key, i * np.uint64(n) + j, p)
    T = np.tril(vals, -1)
    T[np.arange(n), np.arange(n)] = 1
    return T.astype(np.int64)


def planted_support(n: int, r: int, npairs: int, p: int, seed: int):
    """Support of R: a random r-subset of [0, n) (partial Fisher-Yates driven by
    the support stream), its first 2*npairs elements paired consecutively, the
    rest fixed points; every pair / fixed point gets a scaling in [1, p).

    Returns (partner, scale) with partner[i] = j for a pair {i, j}, i for a fixed
    point, -1 outside the support; scale[i] the scaling (0 outside)."""
    assert 0 <= 2 * npairs <= r <= n
    key = derive_key(seed, TAG_SUPPORT)
    skey = derive_key(seed, TAG_SCALE)
    arr = np.arange(n, dtype=np.int64)
    if r > 0:
        rnd = (stream(key, np.arange(r, dtype=np.uint64)) >> np.uint64(32)).astype(np.uint64)
        for k in range(r):
            span = n - k
            j = k + int((int(rnd[k]) * span) >> 32)
            arr[k], arr[j] = arr[j], arr[k]
    sup = arr[:r]
    nfixed = r - 2 * npairs
    scales = 1 + uniform_mod(skey, np.arange(npairs + nfixed, dtype=np.uint64), p - 1) if p > 1 else None
    partner = np.full(n, -1, dtype=np.int64)
    scale = np.zeros(n, dtype=np.int64)
    for q in range(npairs):
        a, b = int(sup[2 * q]), int(sup[2 * q + 1])
        partner[a], partner[b] = b, a
        scale[a] = scale[b] = int(scales[q])
    for f in range(nfixed):
        a = int(sup[2 * npairs + f])
        partner[a] = a
        scale[a] = int(scales[npairs + f])
    return partner, scale


def R_matrix(partner, scale):
    n = len(partner)
    R = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        if partner[i] >= 0:
            R[i, partner[i]] = scale[i]
    return R


def rpm_of_plant(partner):
    """rpm_col of the planted R: partner index or -1 (supp(R) as a rook placement)."""
    return np.asarray(partner, dtype=np.int64).copy()


def _matmul_mod(X, Y, p: int):
    X = np.asarray(X, dtype=np.int64) % p
    Y = np.asarray(Y, dtype=np.int64) % p
    hi, lo = X >> 16, X & 0xFFFF
    out = np.zeros((X.shape[0], Y.shape[1]), dtype=np.int64)
    step = 1 << 15
    for s in range(0, X.shape[1], step):
        ph = (hi[:, s:s + step] @ Y[s:s + step]) % p
        pl = (lo[:, s:s + step] @ Y[s:s + step]) % p
        out = (out + ((ph << 16) % p) + pl) % p
    return out


def planted_matrix(n: int, r: int, npairs: int, p: int, seed: int):
    """A = T R T^T mod p on the host (meant for n up to about a thousand).

    Returns (A as uint32 full symmetric, partner, scale)."""
    partner, scale = planted_support(n, r, npairs, p, seed)
    T = T_matrix(n, p, seed)
    # (T R)[:, partner[k]] gets scale_k * T[:, k]
    TR = np.zeros((n, n), dtype=np.int64)
    for k in range(n):
        if partner[k] >= 0:
            TR[:, partner[k]] = (TR[:, partner[k]] + scale[k] * T[:, k]) % p
    A = _matmul_mod(TR, T.T, p)
    return A.astype(np.uint32), partner, scale


def uniform_symmetric(n: int, p: int, seed: int):
    """Entries i.i.d. uniform in [0, p): A[i, j] = A[j, i] = uniform(key_U, max*n + min)."""
    key = derive_key(seed, TAG_UNIFORM)
    i, j = np.meshgrid(np.arange(n, dtype=np.uint64), np.arange(n, dtype=np.uint64), indexing="ij")
    hi = np.maximum(i, j)
    lo = np.minimum(i, j)
    return uniform_mod(key, hi * np.uint64(n) + lo, p).astype(np.uint32)


def default_pairs(r: int, all_pairs: bool = False) -> int:
    """Pairs in the planted R: floor(r/4) (half of R's non-zeros in 2x2
    transpositions, the rest fixed points) or r/2 with no fixed point."""
    return r // 2 if all_pairs else r // 4


def batch_shapes(count: int, n_lo: int, n_hi: int, seed: int):
    """Orders n_i uniform in [n_lo, n_hi] and ranks r_i uniform in
    [ceil(n_i / 4), n_i] for a batch of `count` matrices (batch stream outputs
    2i and 2i + 1); matrix i is planted with seed ``batch_seed(seed, i)``."""
    key = derive_key(seed, TAG_BATCH)
    u = stream(key, np.arange(2 * count, dtype=np.uint64)) >> np.uint64(32)
    u = u.astype(np.int64)
    n = n_lo + ((u[0::2] * (n_hi - n_lo + 1)) >> 32)
    rlo = (n + 3) // 4
    r = rlo + ((u[1::2] * (n - rlo + 1)) >> 32)
    return n.astype(np.int64), r.astype(np.int64)


def batch_seed(seed: int, i: int) -> int:
    return (int(seed) << 24) + int(i)


# Named workloads: (kind, n, r, p, all_pairs).  Seeds are 180210453 + index.
WORKLOADS = {
    "planted_n256_r192_p65521": ("planted", 256, 192, 65521, False),
    "uniform_n4096_p8388593": ("uniform", 4096, 4096, 8388593, False),
    "planted_n16384_r8192_p67108859": ("planted", 16384, 8192, 67108859, False),
    "planted_n32768_r16384_p2147483647_pairs": ("planted", 32768, 16384, 2147483647, True),
}
# Batch of independent planted matrices: (count, n_lo, n_hi, p); ranks
# uniform in [n/4, n], floor(r/4) pairs each.
BATCH_WORKLOADS = {
    "batch4096_n32to512_p65521": (4096, 32, 512, 65521),
}
SEED_BASE = 180210453
