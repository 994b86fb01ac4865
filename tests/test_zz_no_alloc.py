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


def _run_image(uwb, fn_noalloc, traces, ants, cfg, bf, rule):
    B = traces.shape[0]
    out = torch.empty(B * uwb.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    grid = cfg.grid()
    img = torch.full((B, int(np.prod(grid["n"]))), -1.0, device="cuda")
    if fn_noalloc:
        uwb.uwb_localize_batch_noalloc(traces, ants, grid, cfg.v, cfg.fs, cfg.window, bf, rule,
                                       out, img)
    else:
        ws = torch.empty(uwb.uwb_localize_workspace(B, cfg.n_antennas, cfg.n_samples, grid, bf,
                                                    rule), dtype=torch.uint8, device="cuda")
        uwb.uwb_localize_batch(traces, ants, grid, cfg.v, cfg.fs, cfg.window, bf, rule, ws, out,
                               img)
    torch.cuda.synchronize()
    return [record_to_dict(r) for r in uwb.results_from_device(out)], img.cpu().numpy()


def test_noalloc_smaller_call_after_a_larger_one(uwb):
    """A 6-scan 512 x 512 literal-DMAS call fills more of the shared scratch
    (longer profiles, more boxes) than the 2-scan 64 x 64 DAS call after it:
    the second call, with image output, must read nothing the first left."""
    rule = uwb.uwb_default_rule()
    for name, bf, n in (("dmas2d_512", 2, 6), ("das2d_64", 0, 2)):
        cfg = phantom.CONFIGS[name]
        batch = phantom.make_batch(cfg, n, first_scan=20)
        traces, ants = dev(batch["traces"]), dev(batch["antennas"])
        got, got_img = _run_image(uwb, True, traces, ants, cfg, bf, rule)
        want, want_img = _run_image(uwb, False, traces, ants, cfg, bf, rule)
        for g, w in zip(got, want):
            _same(g, w)
        np.testing.assert_array_equal(got_img, want_img)
    assert uwb.uwb_device_status(clear=True) == 0


def _tiny_case(uwb):
    """An 8 x 8 grid, 2 antennas, 64 samples: about 116 bytes of workspace per
    scan, so the scratch holds a batch of about 145k scans."""
    grid = {"dim": 2, "n": [8, 8, 1], "origin": [-0.0035, -0.0035, 0.0],
            "pitch": [1e-3, 1e-3, 1.0]}
    rule = uwb.uwb_default_rule(mode=uwb.UWB_DECIM_MANUAL, decimation=2, min_segment=2)
    return grid, rule


def test_noalloc_batch_at_the_scratch_limit(uwb):
    """The largest batch whose workspace fits the scratch is accepted and
    gives the workspace entry point's records; one scan more is rejected
    before any device work."""
    grid, rule = _tiny_case(uwb)
    M, N, W, v, fs = 2, 64, 6, 1.0e8, 50.0e9
    need = lambda b: uwb.uwb_localize_workspace(b, M, N, grid, 0, rule)
    lo, hi = 1, 1 << 22
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if 0 < need(mid) <= uwb.NOALLOC_SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid
    B = lo
    assert need(B) <= uwb.NOALLOC_SCRATCH_BYTES < need(B + 1)
    rng = np.random.Generator(np.random.Philox(11))
    traces = torch.from_numpy(rng.standard_normal((B, M, N)).astype(np.float32)).cuda()
    ants = dev(np.array([[0.02, 0.0, 0.0], [-0.015, 0.012, 0.0]], np.float32))
    got = torch.empty(B * uwb.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    uwb.uwb_localize_batch_noalloc(traces, ants, grid, v, fs, W, 0, rule, got)
    ws = torch.empty(need(B), dtype=torch.uint8, device="cuda")
    want = torch.empty_like(got)
    uwb.uwb_localize_batch(traces, ants, grid, v, fs, W, 0, rule, ws, want)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    assert bool((uwb.results_from_device(got)["status"] == 0).all())
    del got, want, ws, traces
    g = uwb.make_grid(grid)
    fake = ctypes.c_void_p(0x1000)   # rejected before any device access
    st = uwb.lib().uwb_localize_batch_noalloc(B + 1, fake, M, N, fake, 0, ctypes.byref(g), v, fs,
                                              W, 0, ctypes.byref(rule), fake, None, None)
    assert st == uwb.UWB_ERR_WORKSPACE
    assert uwb.uwb_device_status(clear=True) == 0
