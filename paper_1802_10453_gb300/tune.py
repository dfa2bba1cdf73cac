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


class OnlineTuner:
    """Introspective schedule choice across a stream of batches (Section 6:
    the threshold is set from experiments with running instances rather than
    fixed a priori).

    Every call factors the caller's batch for real; the schedule it runs with
    is chosen from the times of earlier calls, so no batch is factored twice
    and no extra work is spent on trials.  Outputs never depend on the choice
    (every schedule computes the same exact factorisation).

    Cost model: milliseconds per unit of work, with work = sum of n^3 over the
    batch (known before the call; the ranks are not).  Each candidate keeps an
    exponentially weighted mean of its observed cost.  choose(): a candidate
    never measured is tried first (in the given order); every
    `explore_every`-th call re-measures the candidate measured longest ago, so
    the choice follows a stream whose mix of orders and ranks drifts;
    otherwise the candidate with the lowest mean cost runs.

    Times come from CUDA events on the launching stream and are read without
    blocking: a call's events are taken in once they have completed (at a
    later call, or in flush())."""

    def __init__(self, p: int, candidates=DEFAULT_CANDIDATES, explore_every: int = 8, weight: float = 0.5,
                 path: int = _b.PATH_TC):
        if not candidates:
            raise ValueError("at least one candidate schedule")
        if explore_every < 2:
            raise ValueError("explore_every must be at least 2")
        if not 0.0 < weight <= 1.0:
            raise ValueError("weight must be in (0, 1]")
        self.p = int(p)
        self.path = int(path)
        self.candidates = [tuple(int(v) for v in c) for c in candidates]
        self.explore_every = int(explore_every)
        self.weight = float(weight)
        self.cost = {}       # candidate -> weighted mean ms per unit of work
        self.last_seen = {}  # candidate -> call index of its latest observation
        self.calls = 0
        self.history = []    # (call index, candidate) in launch order
        self._pending = []   # (candidate, work, start event, end event, call index)

    # ---- host logic (no device needed) ----
    def choose(self):
        for c in self.candidates:
            if c not in self.cost and not any(q[0] == c for q in self._pending):
                return c
        measured = [c for c in self.candidates if c in self.cost]
        if not measured:
            return self.candidates[0]
        best = min(measured, key=lambda c: self.cost[c])
        if self.calls % self.explore_every == self.explore_every - 1 and len(measured) > 1:
            others = [c for c in measured if c != best]
            return min(others, key=lambda c: self.last_seen.get(c, -1))
        return best

    def observe(self, cand, ms: float, work: float, call: int | None = None) -> None:
        cand = tuple(cand)
        if work <= 0:
            return
        x = float(ms) / float(work)
        old = self.cost.get(cand)
        self.cost[cand] = x if old is None else (1.0 - self.weight) * old + self.weight * x
        self.last_seen[cand] = self.calls if call is None else call

    def note_launch(self, cand) -> None:
        """Count one call made with `cand` (factor() does this itself)."""
        self.history.append((self.calls, tuple(cand)))
        self.calls += 1

    @property
    def best(self):
        if not self.cost:
            return None
        return min(self.cost, key=self.cost.get)

    # ---- device side ----
    def _collect(self, block: bool) -> None:
        keep = []
        for cand, work, e0, e1, call in self._pending:
            if block:
                e1.synchronize()
            if e1.query():
                self.observe(cand, e0.elapsed_time(e1), work, call)
            else:
                keep.append((cand, work, e0, e1, call))
        self._pending = keep

    def flush(self) -> None:
        """Wait for every timed call and take in its time."""
        self._collect(True)

    def factor(self, batch, stream=None, workspace=None, check: bool = False):
        """Factor `batch` (a binding.Batch) in place with the schedule chosen
        now; returns the status tensor like factor_batched."""
        import torch
        self._collect(False)
        cand = self.choose()
        dev = batch.arena.device
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        work = float(sum(max(n, 0) ** 3 for n in batch.ns))
        _b.set_batched_schedule(*cand)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = _b.factor_batched(batch, self.p, path=self.path, stream=stream, workspace=workspace, check=False)
        e1.record(stream)
        self._pending.append((cand, work, e0, e1, self.calls))
        self.note_launch(cand)
        if check:
            torch.cuda.synchronize(dev)
            bad = int((st != 0).sum().item())
            if bad:
                raise _b.LdltError(int(st[st != 0][0].item()), "%d matrices failed" % bad)
        return st
