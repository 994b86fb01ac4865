"""Progressive re-evaluation on the GPU against the FP64 oracle
(orc_localize_progressive), through the C ABI (needs a GB300). Decisions,
regions, points and locations follow the framework's comparison rules
(tests/parity.py): equal wherever the oracle's own margin exceeds the image
tolerance."""
import numpy as np
import pytest
import torch

import oracle
import phantom
from parity import OracleScan, compare_localize, dev, gpu_localize_batch, record_to_dict

pytestmark = pytest.mark.gpu


def gpu_progressive(uwb, bf, traces, ants, grid, v, fs, W, rule):
    traces = np.asarray(traces, np.float32)
    B, M, N = traces.shape
    ws = torch.empty(uwb.uwb_localize_progressive_workspace(B, M, N, grid, bf, rule),
                     dtype=torch.uint8, device="cuda")
    out = torch.empty(B * uwb.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    uwb.uwb_localize_progressive(dev(traces), dev(ants), grid, v, fs, W, bf, rule, ws, out)
    torch.cuda.synchronize()
    return [record_to_dict(r) for r in uwb.results_from_device(out)]


def _config(name):
    if name == "cube32":   # a 32^3 version of the hemispherical 3-D workload (octree)
        return phantom.with_changes(phantom.CONFIGS["hemi3d_256"], grid_n=(32, 32, 32),
                                    n_antennas=16, n_samples=1024, n_clutter=10)
    return phantom.CONFIGS[name]


@pytest.mark.parametrize("name,bf,n_scans", [("das2d_64", 0, 6), ("dmas2d_512", 0, 4),
                                             ("dmas2d_512", 2, 3), ("cube32", 0, 3),
                                             ("cube32", 2, 2)])
def test_progressive_matches_oracle(gpu, name, bf, n_scans):
    cfg = _config(name)
    b = phantom.make_batch(cfg, n_scans, 40)
    g = cfg.grid()
    ants = b["antennas"].astype(np.float32)
    res = gpu_progressive(gpu, bf, b["traces"], ants, g, cfg.v, cfg.fs, cfg.window,
                          gpu.uwb_default_rule())
    for s in range(n_scans):
        compare_localize(res[s], OracleScan(b["traces"][s], ants, g, cfg.v, cfg.fs, cfg.window,
                                            bf, oracle.make_rule(), progressive=True))


def test_progressive_on_a_full_resolution_lattice_is_the_framework(gpu):
    """Manual decimation D = 1: every region lattice is the region at full
    resolution, the points the framework reads from its profile."""
    cfg = phantom.with_changes(phantom.CONFIGS["das2d_64"], grid_n=(40, 32, 1), extent=0.06)
    b = phantom.make_batch(cfg, 8, 300)
    ants = b["antennas"].astype(np.float32)
    g = cfg.grid()
    rule = gpu.uwb_default_rule(mode=gpu.UWB_DECIM_MANUAL, decimation=1, min_segment=2)
    a = gpu_localize_batch(gpu, 0, b["traces"], ants, g, cfg.v, cfg.fs, cfg.window, rule)
    p = gpu_progressive(gpu, 0, b["traces"], ants, g, cfg.v, cfg.fs, cfg.window, rule)
    for x, y in zip(a, p):
        for k in ("status", "iters", "n_logged", "stop_reason", "roi_lo", "roi_hi", "loc_idx",
                  "child", "box_lo", "box_hi"):
            assert x[k] == y[k], k


def test_progressive_edge_cases(gpu):
    cfg = phantom.CONFIGS["das2d_64"]
    b = phantom.make_batch(cfg, 3, 500)
    tr = b["traces"].copy()
    tr[1] = 0.0                       # no target
    tr[2, 3, 100] = np.nan            # non-finite profile
    res = gpu_progressive(gpu, 0, tr, b["antennas"].astype(np.float32), cfg.grid(), cfg.v,
                          cfg.fs, cfg.window, gpu.uwb_default_rule())
    assert res[0]["status"] == 0 and res[0]["loc_idx"][0] >= 0
    assert res[1]["stop_reason"] == gpu.UWB_STOP_NO_TARGET and res[1]["loc_idx"] == [-1, -1, -1]
    assert res[2]["status"] == gpu.UWB_ERR_NONFINITE
    gpu.uwb_device_status(clear=True)


def test_progressive_replays_in_a_cuda_graph(gpu):
    cfg = phantom.CONFIGS["dmas2d_512"]
    b = phantom.make_batch(cfg, 5, 70)
    tr, ants = dev(b["traces"]), dev(b["antennas"].astype(np.float32))
    g, rule = cfg.grid(), gpu.uwb_default_rule()
    B, M, N = b["traces"].shape
    ws = torch.empty(gpu.uwb_localize_progressive_workspace(B, M, N, g, 2, rule),
                     dtype=torch.uint8, device="cuda")
    direct = torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")

    def run(out, stream=None):
        gpu.uwb_localize_progressive(tr, ants, g, cfg.v, cfg.fs, cfg.window, 2, rule, ws, out,
                                     stream)

    run(direct)
    torch.cuda.synchronize()
    graphed = torch.zeros_like(direct)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        run(graphed, s)
    for _ in range(2):
        graphed.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(graphed, direct)
