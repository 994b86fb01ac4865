"""Ragged batches through the plan API: scans of different antenna counts,
trace lengths, grids and media in one set of launches, traces in float32,
float16 or bfloat16 (needs a GB300)."""
import numpy as np
import pytest
import torch

import oracle
import phantom
from parity import (BF_ORACLE, IMG_TOL, OracleScan, assert_image_close, compare_localize,
                    record_to_dict, rule_pair)

pytestmark = pytest.mark.gpu

TORCH_DT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


def ragged_scans(n=5, seed=0):
    """Scans of one 2-D workload family with different sizes and media."""
    base = phantom.CONFIGS["das2d_64"]
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        cfg = phantom.with_changes(base, n_antennas=int(rng.choice([8, 13, 16, 24])),
                                   n_samples=int(rng.choice([768, 1000, 1024, 1536])),
                                   grid_n=(int(rng.integers(30, 80)), int(rng.integers(30, 80)), 1),
                                   extent=float(rng.uniform(0.08, 0.11)),
                                   eps_r=float(rng.uniform(8.0, 10.0)), n_clutter=5)
        sc = phantom.make_scan(cfg, phantom.BASE_SEED + 900 + k)
        out.append((cfg, sc))
    return out


def plan_for(gpu, scans, dtype, bf, rule):
    specs, host = [], []
    for cfg, sc in scans:
        t = torch.from_numpy(sc["traces"]).cuda().to(TORCH_DT[dtype]).contiguous()
        host.append(t.float().cpu().numpy())        # what the kernels actually read
        specs.append({"traces": t, "antennas": torch.from_numpy(sc["antennas"]).cuda(),
                      "grid": cfg.grid(), "v": cfg.v, "fs": cfg.fs})
    plan = gpu.UwbPlan(specs, scans[0][0].window, bf, rule)
    ws = torch.empty(plan.workspace_bytes(), dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    return plan, host


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("bf", [0, 1, 2])
def test_ragged_images_match_oracle(gpu, dtype, bf):
    scans = ragged_scans()
    g_rule, _ = rule_pair(gpu)
    plan, host = plan_for(gpu, scans, dtype, bf, g_rule)
    imgs = torch.full((plan.image_offset(len(scans)),), -1.0, device="cuda")
    peak = torch.zeros(len(scans), dtype=torch.int64, device="cuda")
    plan.images(imgs, peak)
    torch.cuda.synchronize()
    imgs = imgs.cpu().numpy()
    for k, (cfg, sc) in enumerate(scans):
        g = cfg.grid()
        ref = oracle.image(host[k], sc["antennas"], g, cfg.v, cfg.fs, cfg.window, BF_ORACLE[bf])
        got = imgs[plan.image_offset(k):plan.image_offset(k + 1)].reshape(ref.shape)
        assert_image_close(got, ref, what=f"scan {k} ({dtype})")
        flat = ref.ravel()
        assert abs(flat[int(peak[k])] - flat.max()) <= IMG_TOL * flat.max()
    plan.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bf", [0, 1, 2])
def test_ragged_localize_matches_oracle(gpu, dtype, bf):
    scans = ragged_scans(6, seed=1)
    g_rule, o_rule = rule_pair(gpu)
    plan, host = plan_for(gpu, scans, dtype, bf, g_rule)
    out = torch.empty(len(scans) * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    plan.localize(out)
    torch.cuda.synchronize()
    res = [record_to_dict(r) for r in gpu.results_from_device(out)]
    for k, (cfg, sc) in enumerate(scans):
        compare_localize(res[k], OracleScan(host[k], sc["antennas"], cfg.grid(), cfg.v, cfg.fs,
                                            cfg.window, bf, o_rule))
    plan.close()


def test_benchmark_ragged_batch_sampled_scans_match_oracle(gpu):
    """The benchmark's ragged workload itself: 256 uneven scans (16-96
    antennas, 1024-4096 samples, 128^2-1024^2 grids, clutter) in one plan with
    identity DMAS, float32 traces. Every scan must succeed, and sampled scans
    must match the oracle's decisions, region and location one by one."""
    cfgs = phantom.ragged_configs(256, dim=2)
    scans = [(c, phantom.make_scan(c, phantom.BASE_SEED + 200000 + k)) for k, c in enumerate(cfgs)]
    g_rule, o_rule = rule_pair(gpu)
    plan, host = plan_for(gpu, scans, "f32", 1, g_rule)
    out = torch.empty(len(scans) * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    plan.localize(out)
    torch.cuda.synchronize()
    res = [record_to_dict(r) for r in gpu.results_from_device(out)]
    plan.close()
    assert all(r["status"] == 0 for r in res)
    ties = 0
    for k in (3, 77, 150, 255):
        cfg, sc = scans[k]
        ties += compare_localize(res[k], OracleScan(host[k], sc["antennas"], cfg.grid(), cfg.v,
                                                    cfg.fs, cfg.window, 1, o_rule))["tie"]
    assert ties <= 1, f"{ties} near-ties in 4 sampled scans"


def test_ragged_plan_of_equal_scans_equals_the_uniform_batch(gpu):
    cfg = phantom.CONFIGS["dmas2d_512"]
    batch = phantom.make_batch(cfg, 3)
    g_rule, _ = rule_pair(gpu)
    traces = torch.from_numpy(batch["traces"]).cuda()
    ants = torch.from_numpy(batch["antennas"]).cuda()
    specs = [{"traces": traces[k], "antennas": ants, "grid": cfg.grid(), "v": cfg.v,
              "fs": cfg.fs} for k in range(3)]
    plan = gpu.UwbPlan(specs, cfg.window, 2, g_rule)
    plan.upload(torch.empty(plan.workspace_bytes(), dtype=torch.uint8, device="cuda"))
    a = torch.empty(3 * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    plan.localize(a)
    b = torch.empty_like(a)
    ws = torch.empty(gpu.uwb_localize_workspace(3, cfg.n_antennas, cfg.n_samples, cfg.grid(), 2,
                                                g_rule), dtype=torch.uint8, device="cuda")
    gpu.uwb_localize_batch(traces, ants, cfg.grid(), cfg.v, cfg.fs, cfg.window, 2, g_rule, ws, b)
    torch.cuda.synchronize()
    ra = [record_to_dict(r) for r in gpu.results_from_device(a)]
    rb = [record_to_dict(r) for r in gpu.results_from_device(b)]
    for x, y in zip(ra, rb):
        for key in ("iters", "roi_lo", "roi_hi", "loc_idx", "child", "points_evaluated", "peak"):
            assert x[key] == y[key], key
    plan.close()


@pytest.mark.parametrize("bf", [0, 1])
@pytest.mark.parametrize("window,grid_n", [(20, (45, 37, 1)), (33, (31, 26, 1)),
                                           (20, (18, 14, 11))])
def test_two_points_per_thread_equal_one_point_per_thread(gpu, bf, window, grid_n):
    """Uniform DAS / identity-DMAS batches evaluate two focal points per thread
    as float2 lanes; ragged plans evaluate one per thread. Each lane performs
    the scalar operations in the scalar order, so the images of the same scans
    are bit-identical (ragged tiles, window chunks and a 3-D grid included)."""
    base = phantom.CONFIGS["das2d_64"] if grid_n[2] == 1 else phantom.CONFIGS["hemi3d_256"]
    cfg = phantom.with_changes(base, grid_n=grid_n, window=window, n_antennas=16,
                               n_samples=1024, extent=0.09)
    batch = phantom.make_batch(cfg, 3, 77)
    traces = torch.from_numpy(batch["traces"]).cuda()
    ants = torch.from_numpy(batch["antennas"]).cuda()
    P = int(np.prod(grid_n))
    uni = torch.full((3, P), -1.0, device="cuda")
    gpu.uwb_image_batch(bf, traces, ants, cfg.grid(), cfg.v, cfg.fs, cfg.window, uni)
    g_rule, _ = rule_pair(gpu)
    specs = [{"traces": traces[k], "antennas": ants, "grid": cfg.grid(), "v": cfg.v,
              "fs": cfg.fs} for k in range(3)]
    plan = gpu.UwbPlan(specs, cfg.window, bf, g_rule)
    plan.upload(torch.empty(plan.workspace_bytes(), dtype=torch.uint8, device="cuda"))
    rag = torch.full((plan.image_offset(3),), -2.0, device="cuda")
    plan.images(rag)
    torch.cuda.synchronize()
    assert torch.equal(rag.view(3, P), uni)
    assert bool((uni >= 0).all())
    plan.close()


@pytest.mark.parametrize("bf", [0, 1, 2])
@pytest.mark.parametrize("grid_n", [(45, 37, 1), (64, 32, 1), (18, 14, 11), (16, 8, 8)])
def test_linear_and_shaped_tiles_give_identical_results(gpu, bf, grid_n):
    """The tiling only decides which thread evaluates which focal point:
    images, decimated profiles and localisations are identical with linear
    tiles (the default) and with shaped tiles, exact or ragged on the grid."""
    base = phantom.CONFIGS["das2d_64"] if grid_n[2] == 1 else phantom.CONFIGS["hemi3d_256"]
    cfg = phantom.with_changes(base, grid_n=grid_n, n_antennas=16, n_samples=1024,
                               extent=0.09)
    batch = phantom.make_batch(cfg, 3, 78)
    traces = torch.from_numpy(batch["traces"]).cuda()
    ants = torch.from_numpy(batch["antennas"]).cuda()
    dim = 2 if grid_n[2] == 1 else 3
    shaped = {(2, 2): [16, 8, 1], (2, 3): [8, 4, 4]}.get((bf, dim), [32, 8, 1] if dim == 2
                                                          else [16, 4, 4])
    other = {(2, 2): [32, 4, 1], (2, 3): [16, 4, 2]}.get((bf, dim), [16, 16, 1] if dim == 2
                                                         else [8, 8, 4])
    assert gpu.uwb_tile_shape(bf, dim) == [0, 0, 0]
    g_rule, _ = rule_pair(gpu)
    P = int(np.prod(grid_n))

    def run():
        img = torch.full((3, P), -1.0, device="cuda")
        gpu.uwb_image_batch(bf, traces, ants, cfg.grid(), cfg.v, cfg.fs, cfg.window, img)
        ws = torch.empty(gpu.uwb_localize_workspace(3, cfg.n_antennas, cfg.n_samples,
                                                    cfg.grid(), bf, g_rule),
                         dtype=torch.uint8, device="cuda")
        out = torch.empty(3 * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
        gpu.uwb_localize_batch(traces, ants, cfg.grid(), cfg.v, cfg.fs, cfg.window, bf, g_rule,
                               ws, out)
        torch.cuda.synchronize()
        return img, out

    img0, out0 = run()
    try:
        for tile in (shaped, other):
            gpu.uwb_set_tile_shape(bf, dim, tile)
            img1, out1 = run()
            assert torch.equal(img0, img1), tile
            assert torch.equal(out0, out1), tile
    finally:
        gpu.uwb_set_tile_shape(bf, dim, None)
    assert bool((img0 >= 0).all())


@pytest.mark.parametrize("antennas", [(8, 20, 40, 60), (8, 33, 70, 96)])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_ragged_literal_blocks_per_scan_match_oracle(gpu, dtype, antennas):
    """A literal-DMAS plan holds scans of 8 to 60 antennas (the 64-antenna
    register block: each scan runs the smallest block that holds it, 16, 32 or
    64 antennas, and 16-bit windows land in the per-thread delay table before
    they are widened) or of 8 to 96 (the 96-antenna block form: pairs formed
    block pair by block pair up to each scan's own antenna count, 16-bit
    windows in their own area); images and localisations match the oracle."""
    base = phantom.CONFIGS["das2d_64"]
    scans = []
    for k, m in enumerate(antennas):
        cfg = phantom.with_changes(base, n_antennas=m, grid_n=(40 + 3 * k, 36, 1),
                                   n_samples=1024, n_clutter=5)
        scans.append((cfg, phantom.make_scan(cfg, phantom.BASE_SEED + 950 + k)))
    g_rule, o_rule = rule_pair(gpu)
    plan, host = plan_for(gpu, scans, dtype, 2, g_rule)
    imgs = torch.full((plan.image_offset(len(scans)),), -1.0, device="cuda")
    plan.images(imgs)
    out = torch.empty(len(scans) * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    plan.localize(out)
    torch.cuda.synchronize()
    imgs = imgs.cpu().numpy()
    res = [record_to_dict(r) for r in gpu.results_from_device(out)]
    for k, (cfg, sc) in enumerate(scans):
        g = cfg.grid()
        ref = oracle.image(host[k], sc["antennas"], g, cfg.v, cfg.fs, cfg.window, oracle.DMAS)
        got = imgs[plan.image_offset(k):plan.image_offset(k + 1)].reshape(ref.shape)
        assert_image_close(got, ref, what=f"scan {k} ({cfg.n_antennas} antennas)")
        compare_localize(res[k], OracleScan(host[k], sc["antennas"], g, cfg.v, cfg.fs,
                                            cfg.window, 2, o_rule))
    plan.close()


def test_ragged_localisation_replays_in_a_cuda_graph(gpu):
    scans = ragged_scans(4, seed=2)
    g_rule, _ = rule_pair(gpu)
    plan, _ = plan_for(gpu, scans, "f16", 1, g_rule)
    direct = torch.empty(len(scans) * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    plan.localize(direct)
    torch.cuda.synchronize()
    graphed = torch.zeros_like(direct)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.localize(graphed, stream=s)
    for _ in range(2):
        graphed.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(graphed, direct)
    plan.close()


def test_half_precision_traces_stay_close_to_float32(gpu):
    # the error that 16-bit trace storage adds to each image, against the
    # float64 oracle on the float32 traces
    scans = ragged_scans(3, seed=3)
    g_rule, _ = rule_pair(gpu)
    for dtype, bound in (("f16", 5e-3), ("bf16", 5e-2)):
        plan, _ = plan_for(gpu, scans, dtype, 0, g_rule)
        imgs = torch.empty(plan.image_offset(len(scans)), device="cuda")
        plan.images(imgs)
        torch.cuda.synchronize()
        imgs = imgs.cpu().numpy()
        for k, (cfg, sc) in enumerate(scans):
            ref = oracle.image(sc["traces"], sc["antennas"], cfg.grid(), cfg.v, cfg.fs,
                               cfg.window, oracle.DAS)
            got = imgs[plan.image_offset(k):plan.image_offset(k + 1)].reshape(ref.shape)
            rel = float(np.max(np.abs(got - ref)) / ref.max())
            assert rel < bound, (dtype, k, rel)
        plan.close()


def test_autotune_picks_a_valid_tile_and_keeps_the_results(gpu):
    scans = ragged_scans(4, seed=5)
    g_rule, _ = rule_pair(gpu)
    plan, _ = plan_for(gpu, scans, "f32", 1, g_rule)
    out0 = torch.empty(len(scans) * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    plan.localize(out0)
    ws = torch.empty(plan.workspace_bytes(), dtype=torch.uint8, device="cuda")
    out1 = torch.empty_like(out0)
    try:
        tile, ms = plan.autotune(ws, out1)
        assert tile in ([0, 0, 0], [32, 8, 1], [16, 16, 1], [64, 4, 1], [8, 32, 1]) and ms > 0
        assert gpu.uwb_tile_shape(1, 2) == tile
        plan2, _ = plan_for(gpu, scans, "f32", 1, g_rule)
        out2 = torch.empty_like(out0)
        plan2.localize(out2)
        torch.cuda.synchronize()
        # focal points are computed the same way whatever the tile: same results
        a = [record_to_dict(r) for r in gpu.results_from_device(out0)]
        b = [record_to_dict(r) for r in gpu.results_from_device(out2)]
        for x, y in zip(a, b):
            for key in ("loc_idx", "roi_lo", "roi_hi", "peak", "child"):
                assert x[key] == y[key], key
        plan2.close()
    finally:
        gpu.uwb_set_tile_shape(1, 2, None)
        plan.close()
