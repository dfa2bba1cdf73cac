"""Autotuner of the batched schedule (panel width and cutoff).

The batched kernel is built for a panel width kb in {16, 32, 64}, which fixes
its shared memory and so how many CTAs share an SM; matrices below a cutoff
n_cut may use narrower panels (kb_small).  Which choice is fastest depends on
the batch (orders, ranks, prime), so this module times candidate schedules on
the caller's own batch and keeps the best (Section 6 leaves the threshold
choice to tuning; the update arithmetic is exact, so results never depend on
the choice).  Host logic only: every trial is one ldlt_rpm_factor_batched call.
"""
from __future__ import annotations

from . import binding as _b

# (kb, n_cut, kb_small)
DEFAULT_CANDIDATES = (
    (32, 0, 32),
    (16, 0, 16),
    (64, 0, 64),
    (32, 160, 16),
    (32, 256, 16),
    (64, 256, 32),
)


def tune_batched(batch, p: int, candidates=DEFAULT_CANDIDATES, reps: int = 2, path: int = _b.PATH_TC,
                 workspace=None, apply: bool = True) -> dict:
    """Time each candidate schedule on `batch` (a binding.Batch holding the
    inputs) and return {"best": (kb, n_cut, kb_small), "ms": {cand: ms}}.

    The inputs are saved once and restored before every trial, so the batch
    still holds its inputs on return.  With apply=True the best schedule is
    installed with set_batched_schedule."""
    import torch
    dev = batch.arena.device
    stream = torch.cuda.current_stream(dev)
    saved = batch.arena.clone()
    if workspace is None:
        workspace = torch.empty(_b.batched_workspace_bytes(batch.count, p, path), dtype=torch.uint8,
                                device=dev)
    times = {}
    try:
        for cand in candidates:
            _b.set_batched_schedule(*cand)
            best = None
            for rep in range(reps + 1):  # the first call of a schedule is a warm-up
                batch.arena.copy_(saved)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _b.factor_batched(batch, p, path=path, stream=stream, workspace=workspace, check=False)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if rep:
                    ms = e0.elapsed_time(e1)
                    best = ms if best is None else min(best, ms)
            times[cand] = best
    finally:
        batch.arena.copy_(saved)
        torch.cuda.synchronize(dev)
    choice = min(times, key=times.get)
    _b.set_batched_schedule(*(choice if apply else (32, 0, 32)))
    return {"best": choice, "ms": times}
