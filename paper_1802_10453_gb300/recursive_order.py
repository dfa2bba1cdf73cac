"""The pivot order and block structure of the recursive algorithm (Algorithms
2 and 3, Section 4), read off the rank profile matrix R_A.

Both algorithms reveal R_A (Theorems 1 and 2), and their choices follow from
it alone:
* Algorithm 2 splits the order at m = floor(N/2), orders the leading block's
  pivots by a recursive call, then hands the leading block's non-pivot rows
  (ascending) and the trailing indices to Algorithm 3.
* Algorithm 3 pivots the rows of its off-diagonal block in ascending order,
  each with the column its row holds in R_A (the PLDUQ's pivot: the row's
  leading position after the rows above it), as 2x2 blocks (row, column);
  the remaining columns (ascending) go to Algorithm 2; its non-pivot rows join
  the zero rows.
* 1x1 pivots are the diagonal ones of R_A, met when a recursive call reaches
  a single index; non-pivot rows come last in ascending order.
So one pass of factor (Algorithm 4's order) gives R_A; this module turns it
into the recursion's order, and the given-P mode computes that
factorisation's unique L and D (factor_recursive in binding.py).  Host logic
only, O(n log n).
"""
from __future__ import annotations


def recursive_order(rpm_col):
    """rpm_col[i] = j where (R_A)_ij = 1, else -1.  Returns (perm, starts,
    rank): perm[k] the original index at position k, starts[k] True where a
    2x2 block (k, k+1) starts, rank the number of pivot positions."""
    col = [int(v) for v in rpm_col]
    n = len(col)
    for i, j in enumerate(col):
        if j >= n or (j >= 0 and col[j] != i):
            raise ValueError("rpm_col is not a symmetric rook placement")
    blocks, zeros = _alg2(col, list(range(n)))  # recursion depth about 2 log2(n)
    perm, starts = [], []
    for b in blocks:
        perm += list(b)
        starts += [len(b) == 2] + [False] * (len(b) - 1)
    rank = len(perm)
    perm += zeros
    starts += [False] * len(zeros)
    return perm, starts, rank


def _alg2(col, idx):
    """Algorithm 2 on the indices idx (ascending): (pivot blocks in order,
    non-pivot indices ascending)."""
    N = len(idx)
    if N == 0:
        return [], []
    if N == 1:
        i = idx[0]
        return ([(i,)], []) if col[i] == i else ([], [i])
    m = N // 2
    bA, zA = _alg2(col, idx[:m])
    bB, zB = _alg3(col, zA, idx[m:])
    return bA + bB, sorted(zB)


def _alg3(col, rows, cols):
    """Algorithm 3 on [[0, B], [B^T, C]] with B's rows `rows` and C's indices
    `cols` (both ascending)."""
    if not rows:
        return _alg2(col, cols)
    if not cols:
        return [], list(rows)
    cset = set(cols)
    blocks, used, nonpiv = [], set(), []
    for i in rows:
        j = col[i]
        if j >= 0 and j in cset:
            blocks.append((i, j))
            used.add(j)
        else:
            nonpiv.append(i)
    bZ, zZ = _alg2(col, [j for j in cols if j not in used])
    return blocks + bZ, sorted(zZ + nonpiv)
