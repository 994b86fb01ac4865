"""The no-allocation localisation entry point against the workspace one.

uwb_localize_batch_noalloc serves callers that may not allocate device memory
while they run (fixed-footprint acquisition loops, plug-ins inside a framework
that owns every device allocation): it uses scratch built into the library
instead of a caller workspace. This file runs last so that a stop at the first
failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import phantom
from parity import IMG_TOL, dev, record_to_dict

pytestmark = pytest.mark.gpu


def _run(uwb, fn_noalloc, traces, ants, cfg, bf, rule):
    B = traces.shape[0]
    out = torch.empty(B * uwb.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    grid = cfg.grid()
    if fn_noalloc:
        uwb.uwb_localize_batch_noalloc(traces, ants, grid, cfg.v, cfg.fs, cfg.window, bf, rule,
                                       out)
    else:
        ws = torch.empty(uwb.uwb_localize_workspace(B, cfg.n_antennas, cfg.n_samples, grid, bf,
                                                    rule), dtype=torch.uint8, device="cuda")
        uwb.uwb_localize_batch(traces, ants, grid, cfg.v, cfg.fs, cfg.window, bf, rule, ws, out)
    torch.cuda.synchronize()
    return [record_to_dict(r) for r in uwb.results_from_device(out)]


def _same(a, b):
    for key in ("status", "iters", "n_logged", "stop_reason", "decim", "roi_lo", "roi_hi",
                "loc_idx", "child", "box_lo", "box_hi", "points_evaluated"):
        assert a[key] == b[key], key
    assert abs(a["peak"] - b["peak"]) <= IMG_TOL * max(abs(b["peak"]), 1e-30)
    np.testing.assert_allclose(a["metric_top"], b["metric_top"], rtol=IMG_TOL)


@pytest.mark.parametrize("name,bf", [("das2d_64", 0), ("dmas2d_512", 2)])
def test_noalloc_matches_workspace_entry_point_twice(uwb, name, bf):
    assert torch.cuda.is_available()
    cfg = phantom.CONFIGS[name]
    rule = uwb.uwb_default_rule()
    # two calls in a row on different scans: the second must not see the first's
    # leftovers in the shared scratch
    for first in (0, 6):
        batch = phantom.make_batch(cfg, 6, first_scan=first)
        traces = dev(batch["traces"])
        ants = dev(batch["antennas"])
        want = _run(uwb, False, traces, ants, cfg, bf, rule)
        got = _run(uwb, True, traces, ants, cfg, bf, rule)
        for g, w in zip(got, want):
            _same(g, w)
    assert uwb.uwb_device_status(clear=True) == 0


def test_noalloc_rejects_a_batch_beyond_its_scratch(uwb):
    cfg = phantom.CONFIGS["dmas2d_512"]
    grid = cfg.grid()
    rule = uwb.uwb_default_rule()
    per_scan = uwb.uwb_localize_workspace(1, 32, 2048, grid, 2, rule)
    too_many = uwb.NOALLOC_SCRATCH_BYTES // per_scan * 2
    g = uwb.make_grid(grid)
    fake = ctypes.c_void_p(0x1000)   # rejected before any device access
    st = uwb.lib().uwb_localize_batch_noalloc(too_many, fake, 32, 2048, fake, 0, ctypes.byref(g),
                                              cfg.v, cfg.fs, cfg.window, 2, ctypes.byref(rule),
                                              fake, None, None)
    assert st == uwb.UWB_ERR_WORKSPACE
    assert "scratch" in uwb.uwb_last_error()
