"""GB300 (sm_103a) rank-profile-revealing symmetric factorisation mod p.

Thin Python binding of the C ABI in ``include/ldlt_rpm.h``: argument
marshalling, with every step of the factorisation in the CUDA library
(factor_recursive also derives the recursive algorithms' pivot order from
R_A on the host between two library calls).  PyTorch supplies device memory
and streams.

    import torch, paper_1802_10453_gb300 as lr
    res = lr.factor(A_cuda_uint32_view, p, path=lr.PATH_TC)
    rpm = lr.rpm_from_factor(res)
"""
from .binding import (  # noqa: F401
    PATH_FP64,
    PATH_TC,
    LDLT_OK,
    LDLT_ERR_ARG,
    LDLT_ERR_NOT_PRIME,
    LDLT_ERR_P_RANGE,
    LDLT_ERR_WORKSPACE,
    LDLT_ERR_CUDA,
    LDLT_ERR_TIMEOUT,
    LDLT_ERR_NO_DEVICE,
    LDLT_ERR_TOO_LARGE,
    NOALLOC_MAX_N,
    NOALLOC_BYTES,
    LdltError,
    lib,
    lib_path,
    workspace_bytes,
    factor,
    factor_raw,
    factor_noalloc,
    factor_given,
    factor_recursive,
    given_workspace_bytes,
    factor_batched,
    batched_workspace_bytes,
    set_batched_schedule,
    Batch,
    BATCH_MAX_N,
    rpm_from_factor,
    strict,
    solve,
    trss,
    trss_workspace_bytes,
    LDLT_ERR_INCONSISTENT,
    LDLT_ERR_INTERNAL,
    set_wait_budget_ns,
    set_speculation,
    SPECULATION_DEFAULT,
    test_drop,
    TEST_DROP_SCAN_ANSWERS,
    TEST_DROP_UPDATE_COPIES,
    effective_ops,
)
from .tune import OnlineTuner, tune_batched  # noqa: E402,F401
from .recursive_order import recursive_order  # noqa: E402,F401
