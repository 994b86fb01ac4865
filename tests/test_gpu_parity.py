"""CUDA path against the FP64 oracle, through the C ABI (needs a GB300)."""
import zlib

import numpy as np
import pytest
import torch

import oracle
import phantom
from parity import (BF_ORACLE, IMG_TOL, OracleScan, assert_image_close, compare_localize,
                    dev, record_to_dict, gpu_image_batch, gpu_localize_batch, rule_pair)

pytestmark = pytest.mark.gpu

BFS = [0, 1, 2]  # UWB_DAS, UWB_DMAS, UWB_DMAS_LITERAL


def ring(M, radius, z=0.0, seed=0):
    rng = np.random.default_rng(seed)
    ang = np.sort(rng.uniform(0, 2 * np.pi, M))
    return np.stack([radius * np.cos(ang), radius * np.sin(ang), np.full(M, z)], 1) \
        .astype(np.float32)


def bandlimited(rng, rows, N):
    """Random traces with the UWB pulse's spectrum: white noise filtered by the
    differentiated-Gaussian pulse (6 GHz at 50 GS/s). The float32 delay error
    grows with the delay, and its effect on the image with the trace's slope
    per sample, so stress inputs keep the bandwidth of real echoes."""
    sigma = 50e9 / (2 * np.pi * 6e9)            # pulse sigma in samples
    k = np.arange(-12, 13)
    kern = -(k / sigma) * np.exp(0.5 - 0.5 * (k / sigma) ** 2)
    noise = rng.standard_normal((rows, N + len(k) - 1))
    out = np.stack([np.convolve(r, kern, mode="valid") for r in noise])
    return (out / out.std()).astype(np.float32)


def random_case(M, N, n, extent, W, seed, dim=2, radius=0.07):
    rng = np.random.default_rng(seed)
    tr = bandlimited(rng, M, N)
    if dim == 2:
        ants = ring(M, radius, seed=seed)
    else:
        ants = ring(M, radius, z=0.01, seed=seed)
        ants[:, 2] = rng.uniform(-0.03, 0.03, M)
    pitch = [extent / n[a] if a < dim else 1.0 for a in range(3)]
    origin = [-extent / 2 + pitch[a] / 2 if a < dim else 0.0 for a in range(3)]
    grid = {"dim": dim, "n": list(n), "origin": origin, "pitch": pitch}
    return tr, ants, grid, 1.0e8, 50.0e9, W


CASES = {
    # name: (M, N, grid points, extent [m], W, dim)
    "c1_like": (16, 1024, (64, 64, 1), 0.10, 20, 2),
    "ragged_plain_staging": (5, 1023, (37, 29, 1), 0.09, 7, 2),      # N % 4 != 0
    "window_chunks": (6, 512, (33, 17, 1), 0.08, 33, 2),             # W > 32
    "single_sample_one_antenna": (1, 256, (9, 7, 1), 0.05, 1, 2),
    "literal_register_block_64": (33, 640, (19, 21, 1), 0.08, 5, 2),
    "three_d": (12, 1024, (20, 18, 14), 0.08, 20, 3),
    "window_beyond_shared_memory": (8, 4096, (16, 12, 1), 0.60, 20, 2),  # global-load path
    "literal_block_96": (96, 1024, (23, 19, 1), 0.08, 20, 2),       # three 32-antenna blocks
    "literal_block_70": (70, 1024, (17, 21, 1), 0.08, 9, 2),        # a partial last block
    "block_96_beyond_shared_memory": (80, 4096, (11, 9, 1), 0.60, 20, 2),
}


@pytest.mark.parametrize("bf", BFS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_image_matches_oracle(gpu, case, bf):
    M, N, n, extent, W, dim = CASES[case]
    tr, ants, grid, v, fs, W = random_case(M, N, n, extent, W, seed=zlib.crc32(case.encode()) % 1000, dim=dim)
    img, peak = gpu_image_batch(gpu, bf, tr, ants, grid, v, fs, W)
    ref = oracle.image(tr, ants, grid, v, fs, W, BF_ORACLE[bf])
    assert_image_close(img[0], ref, what=case)
    k = int(np.argmax(ref))
    flat = ref.ravel()
    assert abs(flat[int(peak[0])] - flat[k]) <= IMG_TOL * flat[k]


@pytest.mark.parametrize("bf", BFS)
def test_single_scan_entry_points(gpu, bf):
    M, N, n, extent, W, dim = CASES["c1_like"]
    tr, ants, grid, v, fs, W = random_case(M, N, n, extent, W, seed=5)
    img = torch.zeros(int(np.prod(n)), device="cuda")
    peak = torch.zeros(1, dtype=torch.int64, device="cuda")
    if bf == 0:
        gpu.uwb_das_image(dev(tr), dev(ants), grid, v, fs, W, img, peak)
    else:
        gpu.uwb_dmas_image(dev(tr), dev(ants), grid, v, fs, W, bf == 2, img, peak)
    torch.cuda.synchronize()
    ref = oracle.image(tr, ants, grid, v, fs, W, BF_ORACLE[bf])
    assert_image_close(img.cpu().numpy().reshape(ref.shape), ref)


def test_batched_images_with_per_scan_antennas(gpu):
    M, N, n, extent, W = 10, 512, (21, 23, 1), 0.09, 12
    traces, ants = [], []
    for s in range(3):
        tr, a, grid, v, fs, W = random_case(M, N, n, extent, W, seed=40 + s)
        traces.append(tr)
        ants.append(a)
    traces = np.stack(traces)
    ants = np.stack(ants)
    for bf in BFS:
        img, peak = gpu_image_batch(gpu, bf, traces, ants, grid, v, fs, W)
        for s in range(3):
            ref = oracle.image(traces[s], ants[s], grid, v, fs, W, BF_ORACLE[bf])
            assert_image_close(img[s], ref, what=f"scan {s}")


def test_ragged_trace_with_tma_disabled_by_alignment(gpu):
    # a trace array starting 4 bytes past a 16-byte boundary cannot use TMA
    M, N, n, extent, W = 6, 256, (13, 11, 1), 0.08, 9
    tr, ants, grid, v, fs, W = random_case(M, N, n, extent, W, seed=77)
    buf = torch.zeros(M * N + 1, device="cuda")
    buf[1:] = dev(tr).ravel()
    view = buf[1:].view(M, N)
    img = torch.zeros(int(np.prod(n)), device="cuda")
    gpu.uwb_das_image(view, dev(ants), grid, v, fs, W, img)
    torch.cuda.synchronize()
    ref = oracle.image(tr, ants, grid, v, fs, W, oracle.DAS)
    assert_image_close(img.cpu().numpy().reshape(ref.shape), ref)


# ------------------------------------------------------------------ localisation

def _check_batch(gpu, cfg, bf, seeds, rule_kw=None, ants=None):
    rule_kw = rule_kw or {}
    scans = [phantom.make_scan(cfg, phantom.BASE_SEED + s) for s in seeds]
    traces = np.stack([sc["traces"] for sc in scans])
    ants = scans[0]["antennas"] if ants is None else ants
    grid = cfg.grid()
    g_rule, o_rule = rule_pair(gpu, **rule_kw)
    res = gpu_localize_batch(gpu, bf, traces, ants, grid, cfg.v, cfg.fs, cfg.window, g_rule)
    ties = 0
    for s, sc in enumerate(scans):
        scan = OracleScan(sc["traces"], ants, grid, cfg.v, cfg.fs, cfg.window, bf, o_rule)
        ties += compare_localize(res[s], scan)["tie"]
    assert ties <= max(1, len(seeds) // 4), f"{ties} near-ties in {len(seeds)} scans"
    return res


@pytest.mark.parametrize("bf", BFS)
def test_localize_small_scans(gpu, bf):
    _check_batch(gpu, phantom.CONFIGS["das2d_64"], bf, range(12))


@pytest.mark.parametrize("metric", [1, 2, 3])
def test_localize_other_metrics(gpu, metric):
    _check_batch(gpu, phantom.CONFIGS["das2d_64"], 0, range(6), {"metric": metric})


@pytest.mark.parametrize("bf", [1, 2])
def test_localize_96_antennas(gpu, bf):
    """Localisation with a 96-antenna ring (literal pairs through the
    32-antenna block form; identity DMAS beside it)."""
    cfg = phantom.with_changes(phantom.CONFIGS["das2d_64"], n_antennas=96, radius=0.06)
    _check_batch(gpu, cfg, bf, range(4))


def test_localize_manual_decimation_and_framing(gpu):
    _check_batch(gpu, phantom.CONFIGS["das2d_64"], 1, range(6),
                 {"mode": 0, "decimation": 3, "frame_num": 1, "frame_den": 3, "min_segment": 2})


@pytest.mark.parametrize("bf", [1, 2])
def test_localize_512_grid_with_clutter(gpu, bf):
    # full-size 512 x 512, 32 antennas, 2048 samples, clutter: the launch
    # configuration the benchmark times
    res = _check_batch(gpu, phantom.CONFIGS["dmas2d_512"], bf, range(4))
    for r in res:
        assert r["points_evaluated"] < 512 * 512 / 4


def test_benchmark_batch_sampled_scans_match_oracle(gpu):
    """The benchmark's timed launch itself: 1024 scans of the 512 x 512
    workload (32 antennas, 2048 samples, clutter) in one literal-DMAS batch,
    whose final regions the tile counter splits dynamically. Every scan must
    succeed, and sampled scans must match the oracle's decisions, region and
    location one by one."""
    cfg = phantom.CONFIGS["dmas2d_512"]
    batch = phantom.make_batch(cfg, 1024, first_scan=0)
    grid = cfg.grid()
    g_rule, o_rule = rule_pair(gpu)
    res = gpu_localize_batch(gpu, 2, batch["traces"], batch["antennas"], grid, cfg.v, cfg.fs,
                             cfg.window, g_rule)
    assert all(int(r["status"]) == 0 for r in res)
    ties = 0
    for s in (0, 137, 511, 700, 901, 1023):
        scan = OracleScan(batch["traces"][s], batch["antennas"], grid, cfg.v, cfg.fs,
                          cfg.window, 2, o_rule)
        ties += compare_localize(res[s], scan)["tie"]
    assert ties <= 1, f"{ties} near-ties in 6 sampled scans"


@pytest.mark.parametrize("bf", [0, 1])
def test_packed_selection_batch_matches_oracle(gpu, bf):
    """A batch large enough for the selection kernel's packed form (four scans
    per warp in 8-lane sub-warps, batches of at least 2048 scans of at most
    4096 decimated points): 2050 scans of the 64 x 64 workload, so that the
    last warp holds two scans and two idle sub-warps. A zero scan and a scan
    with a non-finite sample sit in packed warps beside scans that run.
    Sampled scans at every sub-warp position must match the oracle one by
    one; and on every scan the packed form must take the decisions of the
    one-warp-per-scan form (the same batch minus its last three scans)."""
    cfg = phantom.CONFIGS["das2d_64"]
    B = 2050
    batch = phantom.make_batch(cfg, B, first_scan=0)
    traces = batch["traces"].copy()
    traces[1] = 0.0
    traces[6, 3, 100] = np.nan
    ants, grid = batch["antennas"], cfg.grid()
    g_rule, o_rule = rule_pair(gpu)
    packed = gpu_localize_batch(gpu, bf, traces, ants, grid, cfg.v, cfg.fs, cfg.window, g_rule)
    assert packed[1]["stop_reason"] == oracle.STOP_NO_TARGET and packed[1]["status"] == 0
    assert packed[6]["status"] == -4
    assert all(packed[s]["status"] == 0 for s in range(B) if s != 6)
    ties = 0
    for s in (0, 1, 2, 3, 5, 6, 7, 1001, 1234, 2047, 2048, 2049):
        scan = OracleScan(traces[s], ants, grid, cfg.v, cfg.fs, cfg.window, bf, o_rule)
        ties += compare_localize(packed[s], scan)["tie"]
    assert ties <= 2, f"{ties} near-ties in 12 sampled scans"
    # the same scans below the packed form's batch size
    plain = gpu_localize_batch(gpu, bf, traces[:2047], ants, grid, cfg.v, cfg.fs, cfg.window,
                               g_rule)
    differ = []
    for s in range(2047):
        a, b = packed[s], plain[s]
        same = all(a[k] == b[k] for k in ("status", "stop_reason", "iters", "n_logged", "child",
                                          "box_lo", "box_hi", "roi_lo", "roi_hi", "loc_idx"))
        if not same:
            differ.append(s)
            continue
        for k in ("metric_top", "between", "within"):
            np.testing.assert_allclose(a[k], b[k], rtol=1e-12, err_msg=f"scan {s} {k}")
    # decisions may part only where a metric gap or stop margin is at the level
    # of the sums' rounding (about 1e-14)
    for s in differ:
        gaps = [abs(x) for x in plain[s]["metric_gap"] + plain[s]["stop_margin"]]
        assert min(gaps) < 1e-9, f"scan {s}: decisions differ without a near-tie"
    assert len(differ) <= 2


def test_packed_selection_three_d_matches_oracle(gpu):
    """The packed selection in 3-D, where each of a scan's 8 lanes scores one
    of the 8 children alone: 2048 scans of a 32^3 grid (16^3 = 4096 decimated
    points, the packed form's limit), sampled against the oracle and compared
    decision by decision with the one-warp-per-scan form."""
    cfg = phantom.with_changes(phantom.CONFIGS["hemi3d_256"], grid_n=(32, 32, 32),
                               n_antennas=16, n_samples=1024, n_clutter=10)
    B = 2048
    batch = phantom.make_batch(cfg, B, first_scan=0)
    traces, ants, grid = batch["traces"], batch["antennas"], cfg.grid()
    g_rule, o_rule = rule_pair(gpu, min_segment=2)
    packed = gpu_localize_batch(gpu, 0, traces, ants, grid, cfg.v, cfg.fs, cfg.window, g_rule)
    assert packed[0]["dcount"] == [16, 16, 16]
    assert all(r["status"] == 0 for r in packed)
    ties = 0
    for s in (0, 1, 2, 3, 777, 2046, 2047):
        scan = OracleScan(traces[s], ants, grid, cfg.v, cfg.fs, cfg.window, 0, o_rule)
        ties += compare_localize(packed[s], scan)["tie"]
    assert ties <= 2, f"{ties} near-ties in 7 sampled scans"
    plain = gpu_localize_batch(gpu, 0, traces[:B - 1], ants, grid, cfg.v, cfg.fs, cfg.window,
                               g_rule)
    differ = [s for s in range(B - 1)
              if any(packed[s][k] != plain[s][k] for k in ("stop_reason", "iters", "child",
                                                            "box_lo", "box_hi", "loc_idx"))]
    for s in differ:
        gaps = [abs(x) for x in plain[s]["metric_gap"] + plain[s]["stop_margin"]]
        assert min(gaps) < 1e-9, f"scan {s}: decisions differ without a near-tie"
    assert len(differ) <= 2


def test_localize_writes_the_mixed_resolution_image(gpu):
    cfg = phantom.CONFIGS["das2d_64"]
    sc = phantom.make_scan(cfg, phantom.BASE_SEED + 2)
    g_rule, o_rule = rule_pair(gpu)
    grid = cfg.grid()
    res, img = gpu_localize_batch(gpu, 0, sc["traces"], sc["antennas"], grid, cfg.v, cfg.fs,
                                  cfg.window, g_rule, image=True)
    r = res[0]
    full = oracle.image(sc["traces"], sc["antennas"], grid, cfg.v, cfg.fs, cfg.window, oracle.DAS)
    img = img[0]
    written = img >= 0
    # the decimated lattice and the final region are written, nothing else
    D, off = r["decim"], r["offset"]
    expect = np.zeros_like(written)
    expect[0, off[1]::D, off[0]::D] = True
    expect[0, r["roi_lo"][1]:r["roi_hi"][1], r["roi_lo"][0]:r["roi_hi"][0]] = True
    assert np.array_equal(written, expect)
    assert np.max(np.abs(img[written] - full[written])) <= IMG_TOL * full.max()


def test_localize_three_d_small(gpu):
    cfg = phantom.with_changes(phantom.CONFIGS["hemi3d_256"], grid_n=(40, 40, 40),
                               n_antennas=24, n_samples=1024, n_clutter=10)
    for bf in BFS:
        _check_batch(gpu, cfg, bf, range(3), {"min_segment": 2})


def test_localize_edge_cases(gpu):
    cfg = phantom.CONFIGS["das2d_64"]
    grid = cfg.grid()
    good = phantom.make_scan(cfg, phantom.BASE_SEED)
    zero = np.zeros_like(good["traces"])
    nan = good["traces"].copy()
    nan[3, 100] = np.nan
    traces = np.stack([good["traces"], zero, nan, good["traces"]])
    g_rule, o_rule = rule_pair(gpu)
    res = gpu_localize_batch(gpu, 0, traces, good["antennas"], grid, cfg.v, cfg.fs, cfg.window,
                             g_rule)
    for s in range(4):
        compare_localize(res[s], OracleScan(traces[s], good["antennas"], grid, cfg.v, cfg.fs,
                                            cfg.window, 0, o_rule))
    assert res[1]["stop_reason"] == oracle.STOP_NO_TARGET
    assert res[2]["status"] == -4
    assert res[0]["loc_idx"] == res[3]["loc_idx"]


def test_bounded_wait_that_runs_out_is_reported_and_the_context_stays_usable(gpu):
    """Failure detection without a fault: a device wait that nothing completes
    gives up after its probe limit, the kernel records UWB_ERR_TIMEOUT in the
    status word and returns, and the same context then localises as before."""
    assert gpu.uwb_device_status(clear=True) == 0
    gpu.uwb_wait_selftest(4096)
    assert gpu.uwb_device_status(clear=True) == gpu.UWB_ERR_TIMEOUT
    assert gpu.uwb_device_status() == 0
    _check_batch(gpu, phantom.CONFIGS["das2d_64"], 2, range(3))
    assert gpu.uwb_device_status() == 0


def test_localize_degenerate_grids(gpu):
    tr, ants, _, v, fs, W = random_case(4, 256, (1, 1, 1), 0.05, 6, seed=3)
    for n in [(1, 1, 1), (2, 1, 1), (5, 3, 1)]:
        grid = {"dim": 2, "n": list(n), "origin": [0.001, -0.002, 0.0],
                "pitch": [1e-3, 1e-3, 1.0]}
        g_rule, o_rule = rule_pair(gpu, mode=0, decimation=1, min_segment=1)
        res = gpu_localize_batch(gpu, 0, tr, ants, grid, v, fs, W, g_rule)
        compare_localize(res[0], OracleScan(tr, ants, grid, v, fs, W, 0, o_rule))


# ------------------------------------------------------------------ full size

def test_full_resolution_512_literal_dmas(gpu):
    cfg = phantom.CONFIGS["dmas2d_512"]
    scans = [phantom.make_scan(cfg, phantom.BASE_SEED + s) for s in range(2)]
    traces = np.stack([s["traces"] for s in scans])
    ants = scans[0]["antennas"]
    grid = cfg.grid()
    img, peak = gpu_image_batch(gpu, 2, traces, ants, grid, cfg.v, cfg.fs, cfg.window)
    ref = oracle.image(traces[0], ants, grid, cfg.v, cfg.fs, cfg.window, oracle.DMAS)
    assert_image_close(img[0], ref)
    flat = ref.ravel()
    assert abs(flat[int(peak[0])] - flat.max()) <= IMG_TOL * flat.max()
    # second scan: sampled focal points, each computed alone by the oracle
    rng = np.random.default_rng(2)
    pts = rng.integers(0, 512, size=(64, 2))
    ref1 = np.array([oracle.image(traces[1], ants, grid, cfg.v, cfg.fs, cfg.window, oracle.DMAS,
                                  lo=[x, y, 0], cnt=[1, 1, 1])[0, 0, 0] for x, y in pts])
    got1 = np.array([img[1, 0, y, x] for x, y in pts])
    scale = float(img[1].max())
    assert np.max(np.abs(got1 - ref1)) <= IMG_TOL * scale


def test_full_resolution_256_cube_sampled(gpu):
    cfg = phantom.CONFIGS["hemi3d_256"]
    sc = phantom.make_scan(cfg, phantom.BASE_SEED)
    grid = cfg.grid()
    for bf in (0, 1):
        img, peak = gpu_image_batch(gpu, bf, sc["traces"], sc["antennas"], grid, cfg.v, cfg.fs,
                                    cfg.window)
        rng = np.random.default_rng(3 + bf)
        pts = rng.integers(0, 256, size=(48, 3))
        pk = int(peak[0])
        pts = np.vstack([pts, [[pk % 256, (pk // 256) % 256, pk // 65536]]])
        ref = np.array([oracle.image(sc["traces"], sc["antennas"], grid, cfg.v, cfg.fs,
                                     cfg.window, BF_ORACLE[bf], lo=list(p), cnt=[1, 1, 1])[0, 0, 0]
                        for p in pts])
        got = np.array([img[0, z, y, x] for x, y, z in pts])
        assert np.max(np.abs(got - ref)) <= IMG_TOL * float(img[0].max())


def test_localize_256_cube_das(gpu):
    _check_batch(gpu, phantom.CONFIGS["hemi3d_256"], 0, range(1))


# ------------------------------------------------------------------ host-buffer entry point

@pytest.mark.parametrize("name,bf,N,per_scan", [("dmas2d_512", 2, 2048, False),
                                                 ("das2d_64", 1, 1021, False),
                                                 ("das2d_64", 0, 1024, True)])
def test_host_entry_point_matches_device_entry_point(gpu, name, bf, N, per_scan):
    cfg = phantom.with_changes(phantom.CONFIGS[name], n_samples=N)
    batch = phantom.make_batch(cfg, 5)
    grid = cfg.grid()
    ants = batch["antennas"]
    if per_scan:
        rng = np.random.default_rng(9)
        ants = np.stack([ants + rng.normal(0, 1e-3, ants.shape).astype(np.float32)
                         for _ in range(5)])
    g_rule, _ = rule_pair(gpu)
    want = gpu_localize_batch(gpu, bf, batch["traces"], ants, grid, cfg.v, cfg.fs, cfg.window,
                              g_rule)
    tr_h = torch.from_numpy(batch["traces"]).pin_memory()
    an_h = torch.from_numpy(np.ascontiguousarray(ants))
    ws = torch.empty(gpu.uwb_localize_host_workspace(tr_h, an_h, grid, cfg.v, cfg.fs, cfg.window,
                                                     bf, g_rule), dtype=torch.uint8,
                     device="cuda")
    out_h = torch.empty(5 * gpu.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    moved = gpu.uwb_localize_host(tr_h, an_h, grid, cfg.v, cfg.fs, cfg.window, bf, g_rule, ws,
                                  out_h)
    torch.cuda.synchronize()
    got = [record_to_dict(r) for r in out_h.numpy().view(gpu.RESULT_DTYPE)]
    # only the reachable window of the traces crossed the bus
    assert moved < tr_h.numel() * 4
    for g, w in zip(got, want):
        for key in ("status", "iters", "stop_reason", "roi_lo", "roi_hi", "loc_idx", "child",
                    "points_evaluated"):
            assert g[key] == w[key], key
        assert g["peak"] == w["peak"]


# ------------------------------------------------------------------ tumour-presence test

def _small_cube(**kw):
    """A 32^3 version of the hemispherical 3-D workload (16 antennas)."""
    return phantom.with_changes(phantom.CONFIGS["hemi3d_256"], grid_n=(32, 32, 32),
                                n_antennas=16, n_samples=1024, n_clutter=10, **kw)


@pytest.mark.parametrize("name,bf,D2", [("das2d_64", 0, 3), ("dmas2d_512", 2, 20),
                                        ("cube32", 0, 3), ("cube32", 2, 3)])
def test_presence_matches_oracle(gpu, name, bf, D2):
    base = _small_cube() if name == "cube32" else phantom.CONFIGS[name]
    scans, truth = [], []
    for tumor in (True, False):
        cfg = base if tumor else phantom.with_changes(base, n_tumors=(0, 0))
        for s in range(3):
            scans.append(phantom.make_scan(cfg, phantom.BASE_SEED + 700 + s))
    traces = np.stack([sc["traces"] for sc in scans])
    ants = scans[0]["antennas"]
    grid = base.grid()
    g_rule, o_rule = rule_pair(gpu)
    B = len(scans)
    ws = torch.empty(gpu.uwb_presence_workspace(B, base.n_antennas, base.n_samples, grid, bf,
                                                g_rule, D2), dtype=torch.uint8, device="cuda")
    o1 = torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    o2 = torch.empty_like(o1)
    present = torch.full((B,), -1, dtype=torch.int32, device="cuda")
    gpu.uwb_presence_batch(dev(traces), dev(ants), grid, base.v, base.fs, base.window, bf, g_rule,
                           D2, ws, o1, o2, present)
    torch.cuda.synchronize()
    r1 = [record_to_dict(r) for r in gpu.results_from_device(o1)]
    r2 = [record_to_dict(r) for r in gpu.results_from_device(o2)]
    got = present.cpu().numpy()
    o_rule2 = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=D2,
                               min_tumor_diameter=o_rule.min_tumor_diameter, metric=o_rule.metric,
                               min_segment=o_rule.min_segment, frame_num=o_rule.frame_num,
                               frame_den=o_rule.frame_den, max_iters=o_rule.max_iters)
    for s, sc in enumerate(scans):
        want, w1, w2 = oracle.presence(sc["traces"], ants, grid, base.v, base.fs, base.window,
                                       BF_ORACLE[bf], o_rule, D2)
        args = (sc["traces"], ants, grid, base.v, base.fs, base.window, bf)
        t1 = compare_localize(r1[s], OracleScan(*args, o_rule), w1)
        t2 = compare_localize(r2[s], OracleScan(*args, o_rule2), w2)
        # the verdict is the agreement of the two located points
        located = r1[s]["loc_idx"][0] >= 0 and r2[s]["loc_idx"][0] >= 0
        assert bool(got[s]) == (located and r1[s]["loc_idx"] == r2[s]["loc_idx"]), s
        if not (t1["tie"] or t2["tie"]):
            assert bool(got[s]) == want, s
        assert r2[s]["decim"] == D2


# ------------------------------------------------------------------ multistatic

def _ms_gpu_image(gpu, bf, traces, channels, ants, grid, v, fs, W):
    traces = np.asarray(traces, np.float32)
    if traces.ndim == 2:
        traces = traces[None]
    B = traces.shape[0]
    n = list(grid["n"])
    img = torch.full((B, int(np.prod(n))), -1.0, device="cuda")
    peak = torch.zeros(B, dtype=torch.int64, device="cuda")
    gpu.uwb_image_multistatic_batch(bf, dev(traces),
                                    torch.from_numpy(np.ascontiguousarray(channels, np.int32))
                                    .cuda(), dev(ants), grid, v, fs, W, img, peak)
    torch.cuda.synchronize()
    return img.cpu().numpy().reshape(B, n[2], n[1], n[0]), peak.cpu().numpy()


@pytest.mark.parametrize("bf", [0, 1])
def test_multistatic_image_matches_oracle_full_size(gpu, bf):
    cfg = phantom.CONFIGS["ms2d_12"]
    ch = phantom.all_channels(cfg.n_antennas)
    sc = phantom.make_scan(cfg, phantom.BASE_SEED, ch)
    img, peak = _ms_gpu_image(gpu, bf, sc["traces"], ch, sc["antennas"], cfg.grid(), cfg.v,
                              cfg.fs, cfg.window)
    ref = oracle.image_multistatic(sc["traces"], ch, sc["antennas"], cfg.grid(), cfg.v, cfg.fs,
                                   cfg.window, BF_ORACLE[bf])
    assert_image_close(img[0], ref)
    flat = ref.ravel()
    assert abs(flat[int(peak[0])] - flat.max()) <= IMG_TOL * flat.max()


@pytest.mark.parametrize("bf", [0, 1])
@pytest.mark.parametrize("case", ["ragged", "global_path"])
def test_multistatic_image_small_cases(gpu, bf, case):
    M, N, n, extent, W = (5, 1023, (37, 29, 1), 0.09, 7) if case == "ragged" else \
        (4, 4096, (16, 12, 1), 0.60, 20)
    tr, ants, grid, v, fs, W = random_case(M, N, n, extent, W, seed=31)
    rng = np.random.default_rng(32)
    ch = rng.integers(0, M, size=(7, 2)).astype(np.int32)
    trc = bandlimited(rng, 7, N)
    img, _ = _ms_gpu_image(gpu, bf, trc, ch, ants, grid, v, fs, W)
    ref = oracle.image_multistatic(trc, ch, ants, grid, v, fs, W, BF_ORACLE[bf])
    assert_image_close(img[0], ref, what=case)


def test_multistatic_channel_index_out_of_range_is_reported(gpu):
    tr, ants, grid, v, fs, W = random_case(3, 256, (8, 8, 1), 0.05, 4, seed=33)
    ch = np.array([[0, 1], [2, 7]], np.int32)         # antenna 7 does not exist
    gpu.uwb_device_status(clear=True)
    _ms_gpu_image(gpu, 0, tr[:2], ch, ants, grid, v, fs, W)
    assert gpu.uwb_device_status(clear=True) == -1


@pytest.mark.parametrize("bf", [0, 1])
def test_multistatic_localize_matches_oracle(gpu, bf):
    cfg = phantom.CONFIGS["ms2d_12"]
    ch = phantom.all_channels(cfg.n_antennas)
    scans = [phantom.make_scan(cfg, phantom.BASE_SEED + s, ch) for s in range(3)]
    traces = np.stack([sc["traces"] for sc in scans])
    ants = scans[0]["antennas"]
    grid = cfg.grid()
    g_rule, o_rule = rule_pair(gpu)
    B = len(scans)
    ws = torch.empty(gpu.uwb_localize_multistatic_workspace(B, len(ch), cfg.n_samples, grid, bf,
                                                            g_rule), dtype=torch.uint8,
                     device="cuda")
    out = torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    gpu.uwb_localize_multistatic_batch(dev(traces), torch.from_numpy(ch).cuda(), dev(ants), grid,
                                       cfg.v, cfg.fs, cfg.window, bf, g_rule, ws, out)
    torch.cuda.synchronize()
    res = [record_to_dict(r) for r in gpu.results_from_device(out)]
    for s, sc in enumerate(scans):
        compare_localize(res[s], OracleScan(sc["traces"], ants, grid, cfg.v, cfg.fs, cfg.window,
                                            bf, o_rule, channels=ch))


def test_measured_peaks_are_plausible(gpu):
    """uwb_measure_peaks (the denominators of the bench's measured roofline
    fractions): paired-FMA TFLOP/s and conflict-free shared-load wavefronts/s
    on this GPU, between a third of and a little above the derived peaks
    (152 SMs x 128 lanes x 2 FLOP x 2.07 GHz; 1 wavefront per clock per SM)."""
    tflops, wavefronts = gpu.uwb_measure_peaks()
    assert 80.5 / 3 < tflops < 80.5 * 1.1
    assert 314.6e9 / 3 < wavefronts < 314.6e9 * 1.1



@pytest.mark.parametrize("bf", [0, 1])
def test_multistatic_three_d_matches_oracle(gpu, bf):
    """Multistatic (Eq. 2 delays, Eq. 4 over every channel) on a small cube:
    the image and the octree localisation against the oracle."""
    cfg = phantom.with_changes(phantom.CONFIGS["hemi3d_256"], grid_n=(24, 20, 16),
                               n_antennas=8, n_samples=1024, n_clutter=5)
    ch = phantom.all_channels(cfg.n_antennas)
    scans = [phantom.make_scan(cfg, phantom.BASE_SEED + 40 + s, ch) for s in range(2)]
    traces = np.stack([sc["traces"] for sc in scans])
    ants = scans[0]["antennas"]
    grid = cfg.grid()
    img, _ = _ms_gpu_image(gpu, bf, traces, ch, ants, grid, cfg.v, cfg.fs, cfg.window)
    for s, sc in enumerate(scans):
        ref = oracle.image_multistatic(sc["traces"], ch, ants, grid, cfg.v, cfg.fs, cfg.window,
                                       BF_ORACLE[bf])
        assert_image_close(img[s], ref, what=f"3-D multistatic scan {s}")
    g_rule, o_rule = rule_pair(gpu, min_segment=2)
    B = len(scans)
    ws = torch.empty(gpu.uwb_localize_multistatic_workspace(B, len(ch), cfg.n_samples, grid, bf,
                                                            g_rule), dtype=torch.uint8,
                     device="cuda")
    out = torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    gpu.uwb_localize_multistatic_batch(dev(traces), torch.from_numpy(ch).cuda(), dev(ants), grid,
                                       cfg.v, cfg.fs, cfg.window, bf, g_rule, ws, out)
    torch.cuda.synchronize()
    res = [record_to_dict(r) for r in gpu.results_from_device(out)]
    for s, sc in enumerate(scans):
        compare_localize(res[s], OracleScan(sc["traces"], ants, grid, cfg.v, cfg.fs, cfg.window,
                                            bf, o_rule, channels=ch))


@pytest.mark.parametrize("entry", ["localize_das", "localize_literal", "presence",
                                   "multistatic"])
def test_device_entry_points_replay_in_a_cuda_graph(gpu, entry):
    """The device-resident entry points launch kernels only (no host round
    trip, allocation or synchronisation), so a captured CUDA graph replays
    them with byte-identical results."""
    g_rule, _ = rule_pair(gpu)
    if entry == "multistatic":
        cfg = phantom.CONFIGS["ms2d_12"]
        ch = phantom.all_channels(cfg.n_antennas)
        scans = [phantom.make_scan(cfg, phantom.BASE_SEED + 60 + s, ch) for s in range(3)]
        tr = dev(np.stack([sc["traces"] for sc in scans]))
        chd = torch.from_numpy(ch).cuda()
        ants = dev(scans[0]["antennas"])
        bf = 1
        ws = torch.empty(gpu.uwb_localize_multistatic_workspace(3, len(ch), cfg.n_samples,
                                                                cfg.grid(), bf, g_rule),
                         dtype=torch.uint8, device="cuda")
        outs = [torch.empty(3 * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")]

        def run(o, stream=None):
            gpu.uwb_localize_multistatic_batch(tr, chd, ants, cfg.grid(), cfg.v, cfg.fs,
                                               cfg.window, bf, g_rule, ws, o[0],
                                               stream=stream)
    else:
        cfg = phantom.CONFIGS["das2d_64" if entry == "localize_das" else "dmas2d_512"]
        b = phantom.make_batch(cfg, 3, 61)
        tr, ants = dev(b["traces"]), dev(b["antennas"].astype(np.float32))
        bf = 0 if entry == "localize_das" else 2
        B, M, N = b["traces"].shape
        if entry == "presence":
            D2 = 20
            ws = torch.empty(gpu.uwb_presence_workspace(B, M, N, cfg.grid(), bf, g_rule, D2),
                             dtype=torch.uint8, device="cuda")
            outs = [torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda"),
                    torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda"),
                    torch.empty(B, dtype=torch.int32, device="cuda")]

            def run(o, stream=None):
                gpu.uwb_presence_batch(tr, ants, cfg.grid(), cfg.v, cfg.fs, cfg.window, bf,
                                       g_rule, D2, ws, o[0], o[1], o[2], stream=stream)
        else:
            ws = torch.empty(gpu.uwb_localize_workspace(B, M, N, cfg.grid(), bf, g_rule),
                             dtype=torch.uint8, device="cuda")
            outs = [torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")]

            def run(o, stream=None):
                gpu.uwb_localize_batch(tr, ants, cfg.grid(), cfg.v, cfg.fs, cfg.window, bf,
                                       g_rule, ws, o[0], stream=stream)
    run(outs)
    torch.cuda.synchronize()
    graphed = [torch.zeros_like(o) for o in outs]
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        run(graphed, s)
    for _ in range(2):
        for g in graphed:
            g.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for g, o in zip(graphed, outs):
            assert torch.equal(g, o)


@pytest.mark.parametrize("bf", BFS)
def test_exact_tie_scenes_follow_the_gpu_path(gpu, bf):
    """Mirror-symmetric scenes (two equal noiseless scatterers at (+-x, y), the
    symmetric 16-antenna ring, decimation 3 on the 64 x 64 grid, a lattice
    symmetric under x -> 63 - x): the first split's low-x and high-x children
    tie up to rounding, so the GPU may take either. Whichever it takes, the
    oracle replayed along its path must agree on every later step."""
    cfg = phantom.with_changes(phantom.CONFIGS["das2d_64"], snr_db=None)
    ants = phantom.antenna_positions(cfg).astype(np.float32)
    grid = cfg.grid()
    g_rule, o_rule = rule_pair(gpu, mode=0, decimation=3)
    traces = np.stack([phantom.point_scatterer_traces(cfg, [[-x, y, 0], [x, y, 0]], [1, 1])
                       for x, y in ((0.021, 0.013), (0.017, -0.02), (0.03, 0.004),
                                    (0.012, 0.025))])
    res = gpu_localize_batch(gpu, bf, traces, ants, grid, cfg.v, cfg.fs, cfg.window, g_rule)
    for s in range(len(traces)):
        scan = OracleScan(traces[s], ants, grid, cfg.v, cfg.fs, cfg.window, bf, o_rule)
        o = scan.localize()
        assert o["metric_gap"][0] < 1e-9          # the mirror children tie
        compare_localize(res[s], scan, o)
