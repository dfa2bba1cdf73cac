"""Host logic of the online (introspective) schedule tuner: which schedule each
call of a stream runs with, given the times of earlier calls (Section 6: set
the threshold from running instances).  No device is needed: times are fed in
as the device would report them."""
import pytest

from paper_1802_10453_gb300.tune import DEFAULT_CANDIDATES, OnlineTuner


def _run(tuner, true_cost, calls, work=1.0e6):
    """Drive `calls` calls: choose, launch, observe the true cost at once."""
    picks = []
    for _ in range(calls):
        c = tuner.choose()
        tuner.note_launch(c)
        tuner.observe(c, true_cost[c] * work, work)
        picks.append(c)
    return picks


def test_every_candidate_is_tried_once_first_in_order():
    t = OnlineTuner(65521)
    cost = {c: 1.0 + i for i, c in enumerate(DEFAULT_CANDIDATES)}
    picks = _run(t, cost, len(DEFAULT_CANDIDATES))
    assert picks == list(DEFAULT_CANDIDATES)


def test_converges_to_the_fastest_and_mostly_runs_it():
    cands = DEFAULT_CANDIDATES
    cost = {c: 2.0 for c in cands}
    fastest = cands[3]
    cost[fastest] = 1.0
    t = OnlineTuner(65521, explore_every=8)
    picks = _run(t, cost, 200)
    assert t.best == fastest
    tail = picks[len(cands):]
    share = sum(1 for c in tail if c == fastest) / len(tail)
    assert share >= 1.0 - 1.0 / 8 - 0.01
    # exploration visits the others again (the longest unmeasured first)
    assert set(tail) == set(cands)


def test_follows_a_drifting_stream():
    cands = ((32, 0, 32), (16, 0, 16), (64, 0, 64))
    cost = {cands[0]: 1.0, cands[1]: 2.0, cands[2]: 3.0}
    t = OnlineTuner(65521, candidates=cands, explore_every=4, weight=0.5)
    _run(t, cost, 20)
    assert t.best == cands[0]
    # the mix changes: the second schedule becomes the fastest
    cost = {cands[0]: 3.0, cands[1]: 1.0, cands[2]: 3.0}
    picks = _run(t, cost, 4 * len(cands) * 3)
    assert t.best == cands[1]
    assert sum(c == cands[1] for c in picks[-8:]) >= 6


def test_equal_costs_keep_the_first_candidate():
    cands = ((32, 0, 32), (16, 0, 16))
    t = OnlineTuner(65521, candidates=cands, explore_every=3)
    _run(t, {cands[0]: 1.0, cands[1]: 1.0}, 12)
    assert t.best == cands[0]


def test_costs_are_per_unit_of_work():
    cands = ((32, 0, 32), (16, 0, 16))
    t = OnlineTuner(65521, candidates=cands)
    t.observe(cands[0], 10.0, 1.0e6)   # 1e-5 ms per unit
    t.observe(cands[1], 4.0, 1.0e5)    # 4e-5 ms per unit: slower despite the smaller time
    assert t.best == cands[0]
    t.observe(cands[0], 1.0, 0.0)      # no work: ignored
    assert t.cost[cands[0]] == pytest.approx(1.0e-5)


@pytest.mark.parametrize("kw", [dict(candidates=()), dict(explore_every=1), dict(weight=0.0), dict(weight=1.5)])
def test_rejects_bad_arguments(kw):
    with pytest.raises(ValueError):
        OnlineTuner(65521, **kw)
