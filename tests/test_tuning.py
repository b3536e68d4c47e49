"""Host logic of the blocks-per-update autotuner (warmstart.pick_blocks):
the fastest candidate that reaches the target wins, candidates that miss it
are recorded as None, and the best time so far is passed on as a limit."""
import pytest

from paper_1707_05014_gb300 import warmstart as W


def test_fastest_reaching_candidate_wins():
    times = {10: 7020.0, 20: 5100.0, 50: 3430.0, 100: None}
    seen = []

    def trial(b, limit):
        seen.append((b, limit))
        return times[b]

    b, res = W.pick_blocks(trial, (10, 20, 50, 100))
    assert b == 50
    assert res == times
    # each trial gets the best time so far as its limit
    assert seen == [(10, None), (20, 7020.0), (50, 5100.0), (100, 3430.0)]


def test_ties_keep_the_first_candidate_and_misses_are_skipped():
    b, res = W.pick_blocks(lambda b, lim: {4: None, 8: 10.0, 16: 10.0}[b], (4, 8, 16))
    assert b == 8 and res[4] is None


def test_no_candidate_reaching_the_target_is_an_error():
    with pytest.raises(ValueError, match="reached"):
        W.pick_blocks(lambda b, lim: None, (10, 20))
    with pytest.raises(ValueError):
        W.pick_blocks(lambda b, lim: 1.0, ())
    with pytest.raises(ValueError):
        W.pick_blocks(lambda b, lim: 1.0, (0,))
