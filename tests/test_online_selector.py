"""Host logic of the adaptive launch choice of the frame loop's training step
(autotune.OnlineSelector), driven by synthetic step times; no GPU."""
import pytest

from paper_2507_19718_gb300.autotune import OnlineSelector, Trial, drift_candidates


def _run(sel, cost, frames, lag=0):
    """Choose, 'run' and report like the frame loop: the time of a step comes
    back ``lag`` steps later."""
    seq, pending = [], []
    for f in range(frames):
        while len(pending) > lag:
            sel.report(*pending.pop(0))
        i = sel.choose()
        seq.append(i)
        pending.append((i, cost(i, f)))
    return seq


def test_keeps_the_fastest_and_explores_the_others_by_their_gap():
    # gaps 13.8% and 20.7%: the others run at the first rounds, then again
    # after 1 + floor(gap / 5%) rounds, i.e. every 3rd and every 5th round
    sel = OnlineSelector(3, explore_every=4)
    seq = _run(sel, lambda i, f: (2.9, 3.3, 3.5)[i], 48)
    rounds = [seq[k] for k in range(3, 48, 4)]
    assert rounds == [1, 2, 0, 1, 0, 0, 2, 1, 0, 0, 1, 2]
    assert all(seq[k] == 0 for k in range(48) if k % 4 != 3)
    assert sel.current == 0 and sel.switches == 0
    assert sel.runs == [41, 4, 3]


def test_follows_a_drift_of_the_fastest_candidate():
    # the first candidate is fastest on the first 12 steps, the second after
    sel = OnlineSelector(3, explore_every=4)
    cost = lambda i, f: (2.9, 3.3, 3.5)[i] if f < 12 else (3.4, 2.5, 2.9)[i]
    seq = _run(sel, cost, 48, lag=2)
    assert sel.current == 1
    # after the drift the second candidate carries most steps
    assert seq[32:].count(1) >= 12


def test_a_drift_of_the_current_choice_explores_at_once():
    # the current choice slows down by 30% at step 10, right after the
    # regular exploration: every other candidate runs within the next steps
    # instead of waiting for the next regular round
    sel = OnlineSelector(3, explore_every=8)
    cost = lambda i, f: (2.5, 3.0, 3.2)[i] if f < 10 else (3.25, 2.4, 2.7)[i]
    seq = _run(sel, cost, 20, lag=2)
    assert seq[:8] == [0] * 7 + [1]
    assert 1 in seq[10:15] and 2 in seq[10:15]
    assert sel.current == 1 and seq[-3:] == [1, 1, 1]
    # a steady choice never triggers an exploration between regular rounds
    # (the others, 20% and 28% behind, wait 5 and 6 rounds after their first run)
    sel = OnlineSelector(3, explore_every=8)
    assert _run(sel, lambda i, f: (2.5, 3.0, 3.2)[i] * (1 + 0.01 * (f % 3)), 32, lag=2) == \
        [0] * 7 + [1] + [0] * 7 + [2] + [0] * 16


def test_margin_keeps_the_choice_between_near_ties():
    sel = OnlineSelector(2, explore_every=2, margin=0.03)
    _run(sel, lambda i, f: (3.00, 2.95)[i], 40)
    assert sel.current == 0 and sel.switches == 0
    sel = OnlineSelector(2, explore_every=2, margin=0.03)
    _run(sel, lambda i, f: (3.00, 2.80)[i], 40)
    assert sel.current == 1 and sel.switches == 1


def test_single_candidate_and_arguments():
    sel = OnlineSelector(1)
    assert _run(sel, lambda i, f: 1.0, 10) == [0] * 10
    with pytest.raises(ValueError):
        OnlineSelector(0)
    with pytest.raises(ValueError):
        OnlineSelector(2, explore_every=1)


def test_drift_candidates_take_the_next_lower_pixels_per_thread():
    T = lambda tile, cap, q, ms: Trial(tile, 128, cap, q, ms)
    trials = [T((16, 16), 96, 4, 2.88), T((16, 16), 96, 8, 3.21), T((16, 16), 256, 2, 3.30),
              T((8, 32), 128, 2, 3.25), T((16, 16), 256, 1, 3.60), T((8, 8), 512, 1, 3.90)]
    best = trials[0]
    got = drift_candidates(best, trials)
    assert got == [best, trials[3], trials[4]]
    # tuned at one pixel per thread: the only alternative is the next higher
    got = drift_candidates(trials[4], trials)
    assert got == [trials[4], trials[3]]
    assert drift_candidates(best, [best]) == [best]


def test_far_candidates_wait_at_most_eight_rounds_or_for_a_drift():
    # 20% behind: every 5th round; 50% behind: every 8th (the cap)
    sel = OnlineSelector(3, explore_every=4)
    seq = _run(sel, lambda i, f: (2.0, 2.4, 3.0)[i], 4 * 16)
    rounds = [seq[k] for k in range(3, len(seq), 4)]
    assert rounds == [1, 2, 0, 0, 0, 1, 0, 0, 0, 2, 1, 0, 0, 0, 0, 1]
    assert sel.runs == [58, 4, 2] and sel.current == 0
    # a drift of the current choice explores the far candidate at once
    sel = OnlineSelector(3, explore_every=8)
    cost = lambda i, f: (2.0, 2.4, 3.0)[i] if f < 20 else (3.0, 2.9, 2.2)[i]
    seq = _run(sel, cost, 30, lag=1)
    assert 2 in seq[20:26] and sel.current == 2


def test_prior_times_keep_known_slow_candidates_out_of_the_first_rounds():
    # with the autotuner's times the gaps are known from the start (18.5% and
    # 55.6% behind the first measured step): waits of 4 and 8 rounds
    sel = OnlineSelector(3, explore_every=4, prior=[2.9, 3.2, 4.2])
    seq = _run(sel, lambda i, f: (2.7, 3.2, 4.2)[i], 28)
    assert [seq[k] for k in range(3, 28, 4)] == [0, 0, 0, 1, 0, 0, 0]
    assert sel.runs == [27, 1, 0]
    # unknown entries (None, NaN) are measured as before
    sel = OnlineSelector(3, explore_every=4, prior=[None, float("nan"), 4.2])
    assert _run(sel, lambda i, f: (2.7, 3.2, 4.2)[i], 8) == [0, 0, 0, 1, 0, 0, 0, 0]
    with pytest.raises(ValueError):
        OnlineSelector(3, prior=[1.0, 2.0])
