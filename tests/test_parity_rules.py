"""The GPU-vs-oracle comparison rules themselves (tests/parity.py), on the CPU.

Records standing in for the GPU's are made by the oracle along chosen
trajectories. The scene is mirror-symmetric: two equal noiseless point
scatterers at (+-21 mm, 13 mm) seen by the 16-antenna ring, decimation 3 on
the 64 x 64 grid (lattice 0, 3, ..., 63, symmetric under x -> 63 - x). The
first split's low-x and high-x children then score the same up to FP64
rounding: an exact tie, where either child is correct.
"""
import numpy as np
import pytest

import oracle
import phantom
from parity import OracleScan, compare_localize


def _scene():
    cfg = phantom.with_changes(phantom.CONFIGS["das2d_64"], snr_db=None)
    ants = phantom.antenna_positions(cfg).astype(np.float32)
    tr = phantom.point_scatterer_traces(cfg, [[-0.021, 0.013, 0], [0.021, 0.013, 0]], [1, 1])
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=3)
    return OracleScan(tr, ants, cfg.grid(), cfg.v, cfg.fs, cfg.window, 0, rule)


def _record(scan, child=None, cont=None):
    """An oracle result along a forced trajectory, shaped like a GPU record."""
    r = scan.localize(None if child is None else oracle.make_path(child, cont))
    r.pop("path", None)
    return r


def test_own_trajectory_is_accepted_without_ties():
    scan = _scene()
    out = compare_localize(_record(scan), scan)
    assert not out["tie"] and not out["replayed"]


def test_other_child_at_an_exact_tie_is_replayed_and_accepted():
    scan = _scene()
    own = scan.localize()
    assert own["metric_gap"][0] < 1e-12            # the mirror children tie
    other = _record(scan, [own["child"][0] ^ 1])
    assert other["child"][0] != own["child"][0]
    out = compare_localize(other, scan)
    assert out["replayed"] and out["child"] == 1 and out["stop"] == 0


def test_other_child_away_from_a_tie_is_rejected():
    scan = _scene()
    own = scan.localize()
    assert own["metric_gap"][1] > 0.1
    wrong = _record(scan, [-1, own["child"][1] ^ 1])
    assert wrong["status"] == 0
    with pytest.raises(AssertionError, match="child"):
        compare_localize(wrong, scan)


def test_other_stop_outcome_away_from_a_tie_is_rejected():
    scan = _scene()
    own = scan.localize()
    assert own["stop_reason"] == oracle.STOP_METRIC and own["n_logged"] >= 2
    assert abs(own["stop_margin"][1]) > 0.1
    stopped_early = _record(scan, [-1, -1], [-1, 0])
    with pytest.raises(AssertionError, match="stop"):
        compare_localize(stopped_early, scan)


def test_continuation_after_a_tie_is_checked_step_by_step():
    # after the tie at iteration 1, a record that departs again at iteration 2
    # (no tie there) fails, although its first departure alone would pass
    scan = _scene()
    own = scan.localize()
    other = scan.localize(oracle.make_path([own["child"][0] ^ 1]))
    wrong = _record(scan, [own["child"][0] ^ 1, other["child"][1] ^ 1])
    assert wrong["status"] == 0 and other["metric_gap"][1] > 0.1
    with pytest.raises(AssertionError, match="child"):
        compare_localize(wrong, scan)


def test_box_and_location_must_equal_the_oracle():
    scan = _scene()
    good = _record(scan)
    bad_box = dict(good, box_hi=[list(b) for b in good["box_hi"]])
    bad_box["box_hi"][0][0] += 1
    with pytest.raises(AssertionError):
        compare_localize(bad_box, scan)
    # a location one pixel off the peak has a clearly lower energy
    bad_loc = dict(good, loc_idx=[good["loc_idx"][0] + 1] + good["loc_idx"][1:])
    with pytest.raises(AssertionError):
        compare_localize(bad_loc, scan)
