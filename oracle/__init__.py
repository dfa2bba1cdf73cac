"""ORACLE -- test infrastructure only.

A plain CPU statement of what the GPU path computes, written from the paper
(Dumas & Pernet, arXiv 1802.10453).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path never
does.  It shares no code with the CUDA library.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute-force rank profile matrix from Theorem 1, the factor identity of the
abstract, planted rank profiles, closed forms, worked examples of Sections 1
and 2); none is "parity unpinned".
"""
from .oracle import (  # noqa: F401
    build_oracle,
    ldlt_rpm,
    rpm_from_factor,
    rank_mod_p,
    rank_profile_bruteforce,
    canonical_perm_from_rpm,
    check_factor,
    freivalds_check,
    matmul_mod,
    inv_mod,
    max_threads,
    MUTATIONS,
)
