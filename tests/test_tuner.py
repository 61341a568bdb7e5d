"""Host logic of the pool-size tuner (Sec. III, Algorithm 1 restated on
measured throughput) and of the block-shape tuner that follows it, driven by
synthetic throughput curves: no GPU."""
import pytest

from paper_1206_4973_gb300 import build as fsp_build
from paper_1206_4973_gb300 import fsp

UNIT, SMS, MAXP = 256, 152, 152 * 2048


@pytest.fixture(scope="module", autouse=True)
def lib():
    fsp_build.build()
    fsp.load()


def test_doubles_from_sms_blocks_while_improving_then_stops_at_the_limit():
    pools, best = fsp.fsp_tune_simulate(UNIT, SMS, MAXP, lambda p: float(p))
    assert pools[0] == UNIT * SMS
    doubling = [UNIT * SMS * 2**i for i in range(4)]
    assert pools[:4] == doubling  # 38912 .. 311296 = the device limit
    assert best == MAXP
    assert all(UNIT <= q <= MAXP and q % UNIT == 0 for q in pools)


@pytest.mark.parametrize("peak", [60000, 100000, 150000, 250000])
def test_refines_around_a_peaked_curve(peak):
    score = lambda p: 1.0 / (1.0 + abs(p - peak) / peak)  # noqa: E731
    pools, best = fsp.fsp_tune_simulate(UNIT, SMS, MAXP, score)
    tried = set(pools)
    assert best in tried
    assert score(best) == max(score(q) for q in tried)
    assert abs(best - peak) <= 0.35 * peak
    assert len(pools) <= 16


def test_doubles_to_the_limit_even_when_the_score_drops():
    """Algorithm 1 doubles until threads x blocks reaches the device limit and
    keeps the best pool so far; only then does it search around the best."""
    start = UNIT * SMS
    pools, best = fsp.fsp_tune_simulate(UNIT, SMS, MAXP, lambda p: -float(p))
    assert pools[:4] == [start, 2 * start, 4 * start, 8 * start]
    assert best < start  # the refinement found smaller pools better
    assert all(start // 2 <= q <= 2 * start for q in pools[4:])  # the search stays around the best


def test_one_slower_trial_does_not_end_the_doubling():
    """A score that dips once (a noisy measurement at the second pool) and
    peaks at the fourth: the tuner keeps doubling past the dip and settles
    near the peak."""
    start = UNIT * SMS
    peak = 8 * start
    def score(p):
        if p == 2 * start:
            return 0.1  # one slow trial
        return 1.0 / (1.0 + abs(p - peak) / peak)
    pools, best = fsp.fsp_tune_simulate(UNIT, SMS, MAXP, score)
    assert pools[:4] == [start, 2 * start, 4 * start, 8 * start]
    assert best == peak


def test_rejects_bad_arguments():
    with pytest.raises(fsp.FspError):
        fsp.fsp_tune_simulate(0, SMS, MAXP, lambda p: 1.0)


# ------------------------------------------------------- block-shape tuner ---
def test_block_tuner_tries_every_shape_for_a_window_and_keeps_the_fastest():
    scores = [5.0, 9.0, 7.0, 3.0]  # nodes per iteration of shapes 0..3
    cands, best = fsp.fsp_block_tune_simulate(4, 2, lambda c: scores[c])
    # one warm-up iteration on the last shape, then two iterations per shape: 3, 0, 1, 2
    assert cands == [3, 3, 3, 0, 0, 1, 1, 2, 2]
    assert best == 1


def test_block_tuner_ties_keep_the_first_tried_and_one_shape_needs_no_trial():
    cands, best = fsp.fsp_block_tune_simulate(3, 1, lambda c: 4.0)
    assert cands == [2, 2, 0, 1] and best == 2
    assert fsp.fsp_block_tune_simulate(1, 8, lambda c: 1.0) == ([], 0)


def test_block_tuner_rejects_bad_arguments():
    with pytest.raises(fsp.FspError):
        fsp.fsp_block_tune_simulate(0, 8, lambda c: 1.0)
    with pytest.raises(fsp.FspError):
        fsp.fsp_block_tune_simulate(4, 0, lambda c: 1.0)
