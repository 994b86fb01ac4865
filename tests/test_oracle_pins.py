"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
worked example, closed forms, identities between different oracle calls,
invariances and hand-worked cases stored under tests/golden/.
"""
import math

import numpy as np
import pytest

import oracle
import phantom
from conftest import read_golden

V, FS = 1.0e8, 50.0e9          # 1000 samples per metre of one-way path
RNG = np.random.default_rng(1234)


def line_grid(x0, n=1, pitch=1e-3):
    """A 2-D grid whose point (0, 0) sits at (x0, 0)."""
    return {"dim": 2, "n": [n, 1, 1], "origin": [x0, 0.0, 0.0], "pitch": [pitch, 1.0, 1.0]}


def one_point(traces, ants, x, window, bf=oracle.DAS):
    return oracle.image(traces, ants, line_grid(x), V, FS, window, bf)[0, 0, 0]


# ------------------------------------------------------------------ image (Eq. 1, 3)

def test_single_antenna_integer_delay_reads_the_stored_sample():
    # antenna at the origin, focal point 37 mm away: round trip = 74 mm = 37 samples
    tr = RNG.standard_normal((1, 128)).astype(np.float32)
    ant = np.zeros((1, 3), np.float32)
    got = one_point(tr, ant, 0.037, window=1)
    assert got == pytest.approx(float(tr[0, 37]) ** 2, rel=1e-10)


def test_single_antenna_fractional_delay_interpolates_linearly():
    # a linear trace is reproduced exactly by linear interpolation: Y(u) = a + b u
    a, b = 0.25, -0.01
    n = np.arange(128)
    tr = (a + b * n).astype(np.float32)[None, :]
    ant = np.zeros((1, 3), np.float32)
    u = 37.25                                  # 37.25 mm -> 37.25 samples
    got = one_point(tr, ant, u / 1000.0, window=1)
    expect = (float(np.float32(a)) + b * u) ** 2
    assert got == pytest.approx(expect, rel=1e-6)


def test_window_is_centred_on_the_delay():
    # W = 20 samples centred on u (offset -10): for a linear trace
    # I = sum_{k=0}^{19} (a + b (u - 10 + k))^2
    a, b = 1.0, 0.5
    tr = (a + b * np.arange(256)).astype(np.float32)[None, :]
    ant = np.zeros((1, 3), np.float32)
    u = 80.5
    got = one_point(tr, ant, u / 1000.0, window=20)
    expect = sum((a + b * (u - 10 + k)) ** 2 for k in range(20))
    assert got == pytest.approx(expect, rel=1e-9)


def test_samples_outside_the_trace_are_zero():
    tr = RNG.standard_normal((1, 40)).astype(np.float32)
    ant = np.zeros((1, 3), np.float32)
    # u = 3: window covers t = -7 .. 12, samples below 0 are zero
    got = one_point(tr, ant, 0.003, window=20)
    assert got == pytest.approx(float(np.sum(tr[0, 0:13].astype(np.float64) ** 2)), rel=1e-9)
    # u = 35: window t = 25 .. 44, samples from 40 on are zero
    got = one_point(tr, ant, 0.035, window=20)
    assert got == pytest.approx(float(np.sum(tr[0, 25:40].astype(np.float64) ** 2)), rel=1e-9)


def _random_scene(M, N=256, seed=0):
    rng = np.random.default_rng(seed)
    tr = rng.standard_normal((M, N)).astype(np.float32)
    ang = rng.uniform(0, 2 * np.pi, M)
    ants = np.stack([0.06 * np.cos(ang), 0.06 * np.sin(ang), np.zeros(M)], 1).astype(np.float32)
    grid = {"dim": 2, "n": [7, 5, 1], "origin": [-0.01, -0.012, 0.0],
            "pitch": [0.0031, 0.0047, 1.0]}
    return tr, ants, grid


@pytest.mark.parametrize("M", [2, 3, 5, 6])
def test_dmas_single_sample_equals_pair_identity_of_das(M):
    # W = 1: DMAS = (sum_{i<j} x_i x_j)^2 = (((sum x)^2 - sum x^2) / 2)^2, where
    # (sum x)^2 is the all-antenna DAS image and x_i^2 the one-antenna DAS image.
    tr, ants, grid = _random_scene(M, seed=M)
    dmas = oracle.image(tr, ants, grid, V, FS, 1, oracle.DMAS)
    das_all = oracle.image(tr, ants, grid, V, FS, 1, oracle.DAS)
    das_each = sum(oracle.image(tr[i:i + 1], ants[i:i + 1], grid, V, FS, 1, oracle.DAS)
                   for i in range(M))
    expect = ((das_all - das_each) / 2.0) ** 2
    np.testing.assert_allclose(dmas, expect, rtol=1e-9, atol=1e-12 * expect.max())


def _brute_force_image(tr, ants, grid, window, literal_pairs):
    """Eq. 1 and Eq. 3 (DAS) or the Section II.B pair sum (DMAS) written out in
    plain Python loops: round-trip delay 2|r - a_i| fs / v in samples, the
    window centred on it, linear interpolation with zero outside the trace."""
    nx, ny = grid["n"][0], grid["n"][1]
    h = window // 2
    out = np.zeros((1, ny, nx))
    for iy in range(ny):
        for ix in range(nx):
            r = (grid["origin"][0] + ix * grid["pitch"][0], grid["origin"][1] + iy * grid["pitch"][1],
                 grid["origin"][2])
            energy = 0.0
            for k in range(window):
                xs = []
                for i in range(len(ants)):
                    d = math.dist(r, [float(c) for c in ants[i]])
                    t = 2.0 * d * FS / V - h + k
                    n0 = math.floor(t)
                    f = t - n0
                    y0 = float(tr[i][n0]) if 0 <= n0 < tr.shape[1] else 0.0
                    y1 = float(tr[i][n0 + 1]) if 0 <= n0 + 1 < tr.shape[1] else 0.0
                    xs.append((1.0 - f) * y0 + f * y1)
                if literal_pairs:
                    s = sum(xs[i] * xs[j] for i in range(len(xs)) for j in range(i + 1, len(xs)))
                else:
                    s = sum(xs)
                energy += s * s
            out[0, iy, ix] = energy
    return out


@pytest.mark.parametrize("bf", [oracle.DAS, oracle.DMAS])
def test_image_matches_a_brute_force_of_the_definitions(bf):
    # a tiny scene: 3 antennas, a 7 x 5 grid, a 3-sample window
    tr, ants, grid = _random_scene(3, N=256, seed=21)
    got = oracle.image(tr, ants, grid, V, FS, 3, bf)
    want = _brute_force_image(tr, ants, grid, 3, literal_pairs=bf == oracle.DMAS)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12 * want.max())


def test_dmas_two_antennas_is_product_of_single_antenna_energies():
    # M = 2, W = 1: (x_1 x_2)^2 = x_1^2 * x_2^2
    tr, ants, grid = _random_scene(2, seed=11)
    dmas = oracle.image(tr, ants, grid, V, FS, 1, oracle.DMAS)
    e1 = oracle.image(tr[:1], ants[:1], grid, V, FS, 1, oracle.DAS)
    e2 = oracle.image(tr[1:], ants[1:], grid, V, FS, 1, oracle.DAS)
    np.testing.assert_allclose(dmas, e1 * e2, rtol=1e-10)


def _shift(tr, s):
    """Y'[n] = Y[n + s], zero where n + s falls outside the trace."""
    out = np.zeros_like(tr)
    n = tr.shape[1]
    if s >= 0:
        out[:, :n - s] = tr[:, s:]
    else:
        out[:, -s:] = tr[:, :n + s]
    return out


@pytest.mark.parametrize("bf", [oracle.DAS, oracle.DMAS])
@pytest.mark.parametrize("W", [2, 5, 20])
def test_window_sum_equals_sum_of_shifted_single_samples(bf, W):
    # x_i(k) = Y_i(u_i - h + k) = Y'_i(u_i) with Y' shifted by k - h, so the
    # W-sample image is the sum of W one-sample images of shifted traces.
    tr, ants, grid = _random_scene(4, seed=W)
    full = oracle.image(tr, ants, grid, V, FS, W, bf)
    h = W // 2
    parts = sum(oracle.image(_shift(tr, k - h), ants, grid, V, FS, 1, bf) for k in range(W))
    np.testing.assert_allclose(full, parts, rtol=1e-9)


@pytest.mark.parametrize("bf,power", [(oracle.DAS, 2), (oracle.DMAS, 4)])
def test_trace_scaling(bf, power):
    tr, ants, grid = _random_scene(5, seed=3)
    base = oracle.image(tr, ants, grid, V, FS, 6, bf)
    scaled = oracle.image(tr * np.float32(4.0), ants, grid, V, FS, 6, bf)
    np.testing.assert_allclose(scaled, base * 4.0 ** power, rtol=1e-10)


@pytest.mark.parametrize("bf", [oracle.DAS, oracle.DMAS])
def test_antenna_permutation_invariance(bf):
    tr, ants, grid = _random_scene(6, seed=5)
    perm = np.random.default_rng(9).permutation(6)
    a = oracle.image(tr, ants, grid, V, FS, 4, bf)
    b = oracle.image(tr[perm], ants[perm], grid, V, FS, 4, bf)
    np.testing.assert_allclose(a, b, rtol=1e-10)


@pytest.mark.parametrize("bf", [oracle.DAS, oracle.DMAS])
def test_noiseless_point_scatterer_peaks_at_its_own_pixel(bf):
    cfg = phantom.with_changes(phantom.CONFIGS["das2d_64"], snr_db=None)
    g = cfg.grid()
    rng = np.random.default_rng(77)
    for _ in range(4):
        ix, iy = rng.integers(8, 56, size=2)
        p = [g["origin"][0] + ix * g["pitch"][0], g["origin"][1] + iy * g["pitch"][1], 0.0]
        tr = phantom.point_scatterer_traces(cfg, [p], [1.0])
        img = oracle.image(tr, phantom.antenna_positions(cfg).astype(np.float32), g,
                           cfg.v, cfg.fs, cfg.window, bf)
        k = int(np.argmax(img))
        assert (k % 64, k // 64) == (ix, iy)


# ------------------------------------------------------------- decimation (Section III-IV)

def test_automatic_decimation_worked_example():
    gold = read_golden("decimation_worked_example.txt")
    d = float(gold["min_tumor_diameter_m"][0])
    res = float(gold["resolution_m"][0])
    grid = {"dim": 2, "n": [100, 100, 1], "origin": [0, 0, 0], "pitch": [res, res, 1.0]}
    rule = oracle.make_rule(mode=oracle.DECIM_AUTO, min_tumor_diameter=d)
    assert oracle.decimation(rule, grid) == int(gold["decimation"][0])


def test_manual_decimation_is_taken_as_given():
    grid = {"dim": 2, "n": [100, 100, 1], "origin": [0, 0, 0], "pitch": [1e-3, 1e-3, 1.0]}
    for D in (1, 3, 13):
        assert oracle.decimation(oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=D),
                                 grid) == D


@pytest.mark.parametrize("n,D", [(64, 4), (512, 30), (256, 18), (10, 3), (7, 7), (5, 1)])
def test_decimated_lattice_is_centred(n, D):
    o = oracle.lattice_offset(n, D)
    last = o + D * ((n - 1 - o) // D)
    assert 0 <= o < D and last <= n - 1 and n - 1 - last - o in (0, 1)


# ------------------------------------------------------------- Eq. 5, Eq. 6-7

def test_hybrid_metric_limits_stated_in_the_paper():
    mu, var = 0.31, 0.07
    # equal variances in consecutive steps: the mean dominates (is the metric)
    assert oracle.hybrid_metric(mu, var, var) == pytest.approx(mu, rel=1e-15)
    assert oracle.hybrid_metric_unclipped(mu, var, var) == pytest.approx(mu, rel=1e-15)
    # a flat previous region against a dispersed one: the variance dominates
    assert oracle.hybrid_metric(mu, var, 0.0) == pytest.approx(var, rel=1e-15)
    assert oracle.hybrid_metric_unclipped(mu, var, 0.0) == pytest.approx(var, rel=1e-15)
    # a weight halfway: the midpoint of mean and variance
    assert oracle.hybrid_metric(mu, var, var / 2) == pytest.approx((mu + var) / 2, rel=1e-14)
    # a child flatter than its parent: clipped weight 0 -> the mean;
    # the printed formula extrapolates beyond both terms
    assert oracle.hybrid_metric(mu, var, 3 * var) == pytest.approx(mu, rel=1e-15)
    assert oracle.hybrid_metric_unclipped(mu, var, 3 * var) > max(mu, var)


def test_scatter_hand_example():
    gold = read_golden("scatter_hand_example.txt")
    a = [float(x) for x in gold["a"]]
    b = [float(x) for x in gold["b"]]
    w, bb = oracle.scatter(a, b)
    assert w == pytest.approx(float(gold["within"][0]), rel=1e-15)
    assert bb == pytest.approx(float(gold["between"][0]), rel=1e-15)


def test_scatter_decomposes_total_scatter():
    rng = np.random.default_rng(4)
    for _ in range(5):
        a = rng.random(rng.integers(1, 40))
        b = rng.random(rng.integers(1, 40)) * 3
        w, bb = oracle.scatter(a, b)
        pooled = np.concatenate([a, b])
        assert w + bb == pytest.approx(float(np.sum((pooled - pooled.mean()) ** 2)), rel=1e-12)
        w2, b2 = oracle.scatter(a, a + 0.0)
        assert b2 == pytest.approx(0.0, abs=1e-14)


# ------------------------------------------------------------- selection loop (Section III)

def _spike_profile(n, at, D=1):
    e = np.zeros((1, n[1], n[0]))
    e[0, at[1], at[0]] = 1.0
    return e


def test_selection_hand_worked_spike():
    gold = read_golden("select_spike_16x16.txt")
    n = [int(x) for x in gold["grid"]] + [1]
    at = [int(x) for x in gold["spike"]]
    grid = {"dim": 2, "n": n, "origin": [0, 0, 0], "pitch": [1e-3, 1e-3, 1.0]}
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=1,
                            min_segment=int(gold["min_segment"][0]))
    r = oracle.select(_spike_profile(n, at), grid, rule, 1)
    assert r["child"] == [int(x) for x in gold["children"]]
    assert r["box_lo"][0][:2] == [int(x) for x in gold["box1_lo"]]
    assert r["box_hi"][0][:2] == [int(x) for x in gold["box1_hi"]]
    assert r["box_lo"][1][:2] == [int(x) for x in gold["box2_lo"]]
    assert r["box_hi"][1][:2] == [int(x) for x in gold["box2_hi"]]
    assert r["roi_lo"][:2] == [int(x) for x in gold["roi_lo"]]
    assert r["roi_hi"][:2] == [int(x) for x in gold["roi_hi"]]
    assert r["iters"] == int(gold["iters"][0])
    assert r["n_logged"] == int(gold["n_logged"][0])
    assert r["stop_reason"] == int(gold["stop_reason"][0])
    assert r["within"][0] == pytest.approx(float(gold["within1"][0]), rel=1e-12)
    assert r["between"][0] == pytest.approx(float(gold["between1"][0]), rel=1e-6)
    assert r["between"][1] == pytest.approx(float(gold["between2"][0]), rel=1e-6)


def _cube_spike_case():
    gold = read_golden("select_spike_16cube.txt")
    n = [int(x) for x in gold["grid"]]
    at = [int(x) for x in gold["spike"]]
    e = np.zeros((n[2], n[1], n[0]))
    e[at[2], at[1], at[0]] = 1.0
    grid = {"dim": 3, "n": n, "origin": [0, 0, 0], "pitch": [1e-3] * 3}
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=1,
                            min_segment=int(gold["min_segment"][0]))
    return gold, e, grid, rule


def test_selection_hand_worked_spike_in_a_cube():
    """Octree selection (child bit 2 = high z, framing along z, 3-D point counts
    in Eq. 6-7) against a run worked by hand in exact fractions."""
    gold, e, grid, rule = _cube_spike_case()
    r = oracle.select(e, grid, rule, 1)
    blo = [int(x) for x in gold["box_lo"]]
    bhi = [int(x) for x in gold["box_hi"]]
    assert r["child"] == [int(x) for x in gold["children"]]
    assert r["box_lo"] == [blo[3 * i:3 * i + 3] for i in range(len(blo) // 3)]
    assert r["box_hi"] == [bhi[3 * i:3 * i + 3] for i in range(len(bhi) // 3)]
    assert r["roi_lo"] == [int(x) for x in gold["roi_lo"]]
    assert r["roi_hi"] == [int(x) for x in gold["roi_hi"]]
    assert r["iters"] == int(gold["iters"][0])
    assert r["n_logged"] == int(gold["n_logged"][0])
    assert r["stop_reason"] == int(gold["stop_reason"][0])
    np.testing.assert_allclose(r["within"], [float(x) for x in gold["within"]], rtol=1e-13)
    np.testing.assert_allclose(r["between"], [float(x) for x in gold["between"]], rtol=1e-12,
                               atol=1e-18)


def test_selection_cube_is_equivariant_under_axis_swaps():
    """Swapping the y and z axes of the cube's energies swaps child bits 1 and 2
    and the y and z extents of every box (the split points are the same)."""
    gold, e, grid, rule = _cube_spike_case()
    r = oracle.select(e, grid, rule, 1)
    rs = oracle.select(np.ascontiguousarray(np.swapaxes(e, 0, 1)), grid, rule, 1)

    def swap_bits(c):
        return (c & 1) | ((c >> 2) & 1) << 1 | ((c >> 1) & 1) << 2
    assert rs["child"] == [swap_bits(c) for c in r["child"]]
    assert rs["box_lo"] == [[b[0], b[2], b[1]] for b in r["box_lo"]]
    assert rs["box_hi"] == [[b[0], b[2], b[1]] for b in r["box_hi"]]
    assert rs["stop_reason"] == r["stop_reason"] and rs["iters"] == r["iters"]


# ------------------------------------------------------------- trajectory replay (test aid)

def test_replay_without_forcing_is_the_oracle_itself():
    gold, e, grid, rule = _cube_spike_case()
    plain = oracle.select(e, grid, rule, 1)
    free = oracle.select(e, grid, rule, 1, path=oracle.make_path([-1] * 8))
    log = free.pop("path")
    assert free == plain
    assert log["error"] == 0
    assert log["own_child"] == plain["child"] and log["taken_gap"] == [0.0] * 5
    assert log["own_cont"] == [-1, 1, 1, 1, 0]
    own = oracle.select(e, grid, rule, 1, path=oracle.make_path(plain["child"], log["own_cont"]))
    own.pop("path")
    assert own == plain


def test_replay_follows_a_forced_child_and_logs_its_own_choice():
    # 16 x 16 spike of the 2-D hand-worked run: force child 0 (low x, low y) at
    # iteration 1 instead of child 1. Child 0 holds no energy: metric 0, the
    # oracle's own best is child 1, so the gap is 1; the box is child 0's
    # [0,8)^2 grown by 2: [0,10)^2.
    n = [16, 16, 1]
    grid = {"dim": 2, "n": n, "origin": [0, 0, 0], "pitch": [1e-3, 1e-3, 1.0]}
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=1, min_segment=2)
    r = oracle.select(_spike_profile(n, [11, 5]), grid, rule, 1, path=oracle.make_path([0]))
    log = r["path"]
    assert r["child"][0] == 0 and log["own_child"][0] == 1
    assert log["taken_metric"][0] == 0.0 and log["taken_gap"][0] == 1.0
    assert r["box_lo"][0][:2] == [0, 0] and r["box_hi"][0][:2] == [10, 10]
    assert r["metric_top"][0] == 0.0


def test_replay_forced_stop_and_forced_continue():
    gold, e, grid, rule = _cube_spike_case()
    # stop at iteration 2 although Eq. 6-7 says continue: the result is R1
    stop = oracle.select(e, grid, rule, 1, path=oracle.make_path([-1, -1], [-1, 0]))
    assert stop["stop_reason"] == oracle.STOP_METRIC and stop["iters"] == 1
    assert stop["n_logged"] == 2 and stop["path"]["own_cont"][1] == 1
    assert stop["roi_lo"] == [0, 6, 6] and stop["roi_hi"] == [10, 16, 16]
    # continue at iteration 5 although B5 = 0 < B4: the loop goes on from the
    # iteration-5 box [2,7) x [11,15) x [11,15)
    go = oracle.select(e, grid, rule, 1, path=oracle.make_path([-1] * 5, [-1, -1, -1, -1, 1]))
    assert go["path"]["own_cont"][4] == 0
    assert go["n_logged"] > 5 and go["box_lo"][4] == [2, 11, 11]


def test_replay_rejects_a_child_that_is_not_a_candidate():
    # 7 x 8 grid, min_segment 4: the low x half [0,3) is too narrow, so
    # children 0 and 2 are no candidates; child 5 does not exist in 2-D
    n = [7, 8, 1]
    grid = {"dim": 2, "n": n, "origin": [0, 0, 0], "pitch": [1e-3, 1e-3, 1.0]}
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=1, min_segment=4)
    for bad in (0, 2, 5):
        r = oracle.select(_spike_profile(n, [5, 3]), grid, rule, 1, path=oracle.make_path([bad]))
        assert r["path"]["error"] == 1
    ok = oracle.select(_spike_profile(n, [5, 3]), grid, rule, 1, path=oracle.make_path([3]))
    assert ok["path"]["error"] == 0 and ok["child"][0] == 3


ALL_METRICS = [oracle.METRIC_HYBRID, oracle.METRIC_MEAN, oracle.METRIC_VARIANCE,
               oracle.METRIC_HYBRID_UNCLIPPED]


@pytest.mark.parametrize("metric", ALL_METRICS)
def test_selection_keeps_a_lone_spike(metric):
    # zero energy everywhere but one point: only the child holding it has a
    # non-zero mean and variance, so every metric must keep it
    n = [64, 64, 1]
    grid = {"dim": 2, "n": n, "origin": [0, 0, 0], "pitch": [1e-3, 1e-3, 1.0]}
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=1, metric=metric,
                            min_segment=2, max_iters=12)
    rng = np.random.default_rng(8)
    for _ in range(6):
        at = rng.integers(0, 64, size=2)
        r = oracle.select(_spike_profile(n, at), grid, rule, 1)
        assert r["n_logged"] >= 1
        for lo, hi in zip(r["box_lo"], r["box_hi"]):
            assert lo[0] <= at[0] < hi[0] and lo[1] <= at[1] < hi[1]
        assert r["roi_lo"][0] <= at[0] < r["roi_hi"][0]
        assert r["roi_lo"][1] <= at[1] < r["roi_hi"][1]


@pytest.mark.parametrize("metric", ALL_METRICS)
def test_selection_mirrors_with_the_profile(metric):
    # reflecting the energies in x reflects every choice (child bit 0 flips),
    # as long as every split is symmetric: the first two regions have even sides
    n = [64, 64, 1]
    grid = {"dim": 2, "n": n, "origin": [0, 0, 0], "pitch": [1e-3, 1e-3, 1.0]}
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=1, metric=metric,
                            max_iters=2)
    rng = np.random.default_rng(18)
    for _ in range(6):
        base = rng.random((1, 64, 64)) ** 4
        r = oracle.select(base, grid, rule, 1)
        rm = oracle.select(base[:, :, ::-1].copy(), grid, rule, 1)
        assert [c ^ 1 for c in r["child"]] == rm["child"]
        assert r["stop_reason"] == rm["stop_reason"] and r["iters"] == rm["iters"]
        for lo, hi, lom, him in zip(r["box_lo"], r["box_hi"], rm["box_lo"], rm["box_hi"]):
            assert (lom[0], him[0]) == (64 - hi[0], 64 - lo[0])
            assert (lom[1], him[1]) == (lo[1], hi[1])


def test_selection_stops_when_no_child_is_large_enough():
    n = [8, 8, 1]
    grid = {"dim": 2, "n": n, "origin": [0, 0, 0], "pitch": [1e-3, 1e-3, 1.0]}
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=1, min_segment=5)
    r = oracle.select(_spike_profile(n, [2, 3]), grid, rule, 1)
    assert r["stop_reason"] == oracle.STOP_MINSIZE and r["iters"] == 0
    assert r["roi_lo"][:2] == [0, 0] and r["roi_hi"][:2] == [8, 8]


def test_selection_iteration_cap():
    n = [64, 64, 1]
    grid = {"dim": 2, "n": n, "origin": [0, 0, 0], "pitch": [1e-3, 1e-3, 1.0]}
    e = np.zeros((1, 64, 64))
    e[0, 30, 40] = 1.0
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=1, max_iters=1)
    r = oracle.select(e, grid, rule, 1)
    assert r["stop_reason"] == oracle.STOP_CAP and r["iters"] == 1
    assert r["roi_lo"] == r["box_lo"][0] and r["roi_hi"] == r["box_hi"][0]


# ------------------------------------------------------------- whole method

def test_scaling_the_traces_changes_no_decision():
    cfg = phantom.CONFIGS["das2d_64"]
    sc = phantom.make_scan(cfg, phantom.BASE_SEED + 3)
    g = cfg.grid()
    a = oracle.localize(sc["traces"], sc["antennas"], g, cfg.v, cfg.fs, cfg.window, oracle.DMAS)
    b = oracle.localize(sc["traces"] * np.float32(8.0), sc["antennas"], g, cfg.v, cfg.fs,
                        cfg.window, oracle.DMAS)
    for key in ("child", "box_lo", "box_hi", "roi_lo", "roi_hi", "loc_idx", "iters",
                "stop_reason"):
        assert a[key] == b[key]


@pytest.mark.parametrize("bf", [oracle.DAS, oracle.DMAS])
def test_no_accuracy_loss_on_noiseless_single_scatterers(bf):
    # the paper's claim: the framework finds the location the full-resolution
    # beamformer finds
    cfg = phantom.with_changes(phantom.CONFIGS["das2d_64"], snr_db=None)
    g = cfg.grid()
    for s in range(8):
        sc = phantom.make_scan(cfg, phantom.BASE_SEED + 100 + s)
        full = oracle.image(sc["traces"], sc["antennas"], g, cfg.v, cfg.fs, cfg.window, bf)
        k = int(np.argmax(full))
        r = oracle.localize(sc["traces"], sc["antennas"], g, cfg.v, cfg.fs, cfg.window, bf)
        assert r["loc_idx"][:2] == [k % 64, k // 64]
        assert r["points_evaluated"] < 64 * 64


def test_all_zero_traces_report_no_target():
    cfg = phantom.CONFIGS["das2d_64"]
    tr = np.zeros((cfg.n_antennas, cfg.n_samples), np.float32)
    r = oracle.localize(tr, phantom.antenna_positions(cfg), cfg.grid(), cfg.v, cfg.fs,
                        cfg.window, oracle.DAS)
    assert r["status"] == 0 and r["stop_reason"] == oracle.STOP_NO_TARGET
    assert r["loc_idx"] == [-1, -1, -1]


def test_nonfinite_trace_is_reported():
    cfg = phantom.CONFIGS["das2d_64"]
    sc = phantom.make_scan(cfg, phantom.BASE_SEED)
    tr = sc["traces"].copy()
    tr[:, :] = np.nan
    r = oracle.localize(tr, sc["antennas"], cfg.grid(), cfg.v, cfg.fs, cfg.window, oracle.DAS)
    assert r["status"] == -4


def test_three_d_localisation_runs_on_a_small_cube():
    cfg = phantom.with_changes(phantom.CONFIGS["hemi3d_256"], grid_n=(24, 24, 24),
                               n_antennas=12, n_samples=1024, snr_db=None, n_clutter=0,
                               n_tumors=(1, 1), tumor_amp=(1.0, 1.0))
    sc = phantom.make_scan(cfg, phantom.BASE_SEED)
    g = cfg.grid()
    full = oracle.image(sc["traces"], sc["antennas"], g, cfg.v, cfg.fs, cfg.window, oracle.DAS)
    k = int(np.argmax(full))
    r = oracle.localize(sc["traces"], sc["antennas"], g, cfg.v, cfg.fs, cfg.window, oracle.DAS,
                        oracle.make_rule(min_segment=2))
    assert r["loc_idx"] == [k % 24, (k // 24) % 24, k // 576]
    assert all(0 <= c < 8 for c in r["child"])


# ------------------------------------------------------------- tumour-presence test (Section IV)

def test_presence_with_the_same_factor_twice_confirms_any_located_target():
    cfg = phantom.CONFIGS["das2d_64"]
    sc = phantom.make_scan(cfg, phantom.BASE_SEED + 7)
    rule = oracle.make_rule()
    D = oracle.decimation(rule, cfg.grid())
    present, r1, r2 = oracle.presence(sc["traces"], sc["antennas"], cfg.grid(), cfg.v, cfg.fs,
                                      cfg.window, oracle.DAS, rule, D)
    assert present and r1["loc_idx"] == r2["loc_idx"] and r2["decim"] == D


def test_presence_is_declined_without_any_echo():
    cfg = phantom.CONFIGS["das2d_64"]
    tr = np.zeros((cfg.n_antennas, cfg.n_samples), np.float32)
    present, r1, _ = oracle.presence(tr, phantom.antenna_positions(cfg), cfg.grid(), cfg.v,
                                     cfg.fs, cfg.window, oracle.DAS, oracle.make_rule(), 3)
    assert not present and r1["stop_reason"] == oracle.STOP_NO_TARGET


def test_presence_reports_disagreeing_runs():
    # two point scatterers of equal strength far apart: decimation factors that
    # sample them differently may send the search to different ones; whenever
    # the two runs' locations differ the verdict must be "absent"
    cfg = phantom.with_changes(phantom.CONFIGS["das2d_64"], snr_db=None)
    g = cfg.grid()
    for D2 in (2, 3, 5):
        tr = phantom.point_scatterer_traces(cfg, [[-0.02, -0.01, 0], [0.021, 0.012, 0]], [1, 1])
        present, r1, r2 = oracle.presence(tr, phantom.antenna_positions(cfg), g, cfg.v, cfg.fs,
                                          cfg.window, oracle.DAS, oracle.make_rule(), D2)
        assert present == (r1["loc_idx"] == r2["loc_idx"])


# ------------------------------------------------------------- multistatic (Eq. 2, Eq. 4)

def test_diagonal_channels_reproduce_the_monostatic_image():
    tr, ants, grid = _random_scene(5, seed=21)
    diag = np.stack([np.arange(5), np.arange(5)], 1)
    for bf in (oracle.DAS, oracle.DMAS):
        mono = oracle.image(tr, ants, grid, V, FS, 6, bf)
        ms = oracle.image_multistatic(tr, diag, ants, grid, V, FS, 6, bf)
        np.testing.assert_allclose(ms, mono, rtol=1e-12)


def test_single_channel_delay_is_transmitter_plus_receiver_path():
    # tx at the origin, rx at (30 mm, 0): the focal point (0, 40 mm) is 40 mm
    # from tx and 50 mm from rx, so u = 90 mm of path * 500 samples/m = 45
    a, b = 0.5, 0.02
    tr = (a + b * np.arange(128)).astype(np.float32)[None, :]
    ants = np.array([[0, 0, 0], [0.03, 0, 0]], np.float32)
    grid = {"dim": 2, "n": [1, 1, 1], "origin": [0.0, 0.04, 0.0], "pitch": [1e-3, 1e-3, 1.0]}
    got = oracle.image_multistatic(tr, [[0, 1]], ants, grid, V, FS, 1)[0, 0, 0]
    assert got == pytest.approx((a + b * 45.0) ** 2, rel=1e-6)


def test_multistatic_dmas_single_sample_identity():
    tr, ants, grid = _random_scene(4, seed=22)
    rng = np.random.default_rng(3)
    ch = rng.integers(0, 4, size=(6, 2))
    trc = rng.standard_normal((6, 256)).astype(np.float32)
    dmas = oracle.image_multistatic(trc, ch, ants, grid, V, FS, 1, oracle.DMAS)
    das = oracle.image_multistatic(trc, ch, ants, grid, V, FS, 1, oracle.DAS)
    each = sum(oracle.image_multistatic(trc[c:c + 1], ch[c:c + 1], ants, grid, V, FS, 1)
               for c in range(6))
    np.testing.assert_allclose(dmas, ((das - each) / 2) ** 2, rtol=1e-9,
                               atol=1e-12 * dmas.max())


def test_reciprocal_channels_have_the_same_delay():
    tr, ants, grid = _random_scene(3, seed=23)
    one = tr[:1]
    a = oracle.image_multistatic(one, [[0, 2]], ants, grid, V, FS, 5)
    b = oracle.image_multistatic(one, [[2, 0]], ants, grid, V, FS, 5)
    np.testing.assert_array_equal(a, b)


def test_multistatic_localisation_with_diagonal_channels_is_monostatic():
    cfg = phantom.CONFIGS["das2d_64"]
    sc = phantom.make_scan(cfg, phantom.BASE_SEED + 4)
    diag = np.stack([np.arange(cfg.n_antennas)] * 2, 1)
    g = cfg.grid()
    mono = oracle.localize(sc["traces"], sc["antennas"], g, cfg.v, cfg.fs, cfg.window, oracle.DAS)
    ms = oracle.localize_multistatic(sc["traces"], diag, sc["antennas"], g, cfg.v, cfg.fs,
                                     cfg.window, oracle.DAS)
    for key in ("child", "box_lo", "box_hi", "roi_lo", "roi_hi", "loc_idx", "iters"):
        assert ms[key] == mono[key]


def test_multistatic_scene_locates_its_tumour():
    cfg = phantom.with_changes(phantom.CONFIGS["ms2d_12"], snr_db=None, n_clutter=0,
                               grid_n=(96, 96, 1))
    ch = phantom.all_channels(cfg.n_antennas)
    sc = phantom.make_scan(cfg, phantom.BASE_SEED + 1, ch)
    g = cfg.grid()
    r = oracle.localize_multistatic(sc["traces"], ch, sc["antennas"], g, cfg.v, cfg.fs,
                                    cfg.window, oracle.DAS)
    assert np.linalg.norm(np.array(r["loc_xyz"]) - sc["tumors"][0]) < 2 * g["pitch"][0]


# ------------------------------------------------- progressive re-evaluation (variant)

@pytest.mark.parametrize("lo,hi,c0,want", [
    (0, 512, 18, (9, 29, 18)),     # step ceil(512/18) = 29; (511 mod 29) // 2 = 9
    (128, 320, 18, (130, 11, 18)),  # side 192: step 11, (191 mod 11) // 2 = 2
    (5, 21, 18, (5, 1, 16)),        # a side below c0 is imaged at full resolution
    (0, 37, 18, (0, 3, 13)),
])
def test_region_lattice_hand_values(lo, hi, c0, want):
    assert oracle.region_lattice(lo, hi, c0) == want


def test_region_lattice_stays_inside_and_below_the_count():
    rng = np.random.default_rng(5)
    for _ in range(500):
        lo = int(rng.integers(0, 300))
        hi = lo + int(rng.integers(1, 400))
        c0 = int(rng.integers(1, 40))
        first, step, cnt = oracle.region_lattice(lo, hi, c0)
        last = first + step * (cnt - 1)
        assert lo <= first and last < hi and cnt <= c0 and step >= 1
        # one more point would leave the range, and the lattice is centred
        assert last + step >= hi
        assert abs((first - lo) - (hi - 1 - last)) <= step


def _scene_for_progressive(seed, n=(24, 20), M=6):
    rng = np.random.default_rng(seed)
    ang = np.sort(rng.uniform(0, 2 * np.pi, M))
    ants = np.stack([0.05 * np.cos(ang), 0.05 * np.sin(ang), np.zeros(M)], 1).astype(np.float32)
    pitch = 0.06 / n[0]
    grid = {"dim": 2, "n": [n[0], n[1], 1], "origin": [-0.03 + pitch / 2, -0.025, 0.0],
            "pitch": [pitch, pitch, 1.0]}
    pts = [[rng.uniform(-0.02, 0.02), rng.uniform(-0.015, 0.015), 0.0]]
    cfg = phantom.with_changes(phantom.CONFIGS["das2d_64"], n_antennas=M, snr_db=None)
    tr = phantom.synthesize(cfg, np.array(pts), np.array([1.0]), np.array([cfg.eps_r]),
                            ants.astype(np.float64)).astype(np.float32)
    tr += rng.normal(0, 0.05, tr.shape).astype(np.float32)
    return tr, ants, grid, cfg


SAME_KEYS = ("status", "iters", "n_logged", "stop_reason", "roi_lo", "roi_hi", "loc_idx",
             "child", "n_children", "box_lo", "box_hi")


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("bf", [oracle.DAS, oracle.DMAS])
def test_progressive_on_a_full_resolution_lattice_is_the_paper_method(seed, bf):
    # D = 1: every region lattice is the region at full resolution, the same
    # points the paper's loop reads from its (full-resolution) profile
    tr, ants, grid, cfg = _scene_for_progressive(seed)
    rule = oracle.make_rule(mode=oracle.DECIM_MANUAL, decimation=1, min_segment=2)
    a = oracle.localize(tr, ants, grid, cfg.v, cfg.fs, cfg.window, bf, rule)
    b = oracle.localize_progressive(tr, ants, grid, cfg.v, cfg.fs, cfg.window, bf, rule)
    for k in SAME_KEYS:
        assert a[k] == b[k], k
    np.testing.assert_allclose(b["metric_top"], a["metric_top"], rtol=1e-12)
    np.testing.assert_allclose(b["between"], a["between"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b["within"], a["within"], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_progressive_first_iteration_is_the_paper_method(seed):
    cfg = phantom.CONFIGS["dmas2d_512"]
    cfg = phantom.with_changes(cfg, grid_n=(96, 96, 1), extent=0.08)
    sc = phantom.make_scan(cfg, phantom.BASE_SEED + 70 + seed)
    rule = oracle.make_rule(max_iters=1)
    a = oracle.localize(sc["traces"], sc["antennas"], cfg.grid(), cfg.v, cfg.fs, cfg.window,
                        oracle.DAS, rule)
    b = oracle.localize_progressive(sc["traces"], sc["antennas"], cfg.grid(), cfg.v, cfg.fs,
                                    cfg.window, oracle.DAS, rule)
    for k in SAME_KEYS + ("points_evaluated",):
        assert a[k] == b[k], k


def test_progressive_points_are_the_lattices_it_imaged():
    cfg = phantom.with_changes(phantom.CONFIGS["dmas2d_512"], grid_n=(128, 128, 1), extent=0.08)
    sc = phantom.make_scan(cfg, phantom.BASE_SEED + 91)
    g = cfg.grid()
    r = oracle.localize_progressive(sc["traces"], sc["antennas"], g, cfg.v, cfg.fs, cfg.window,
                                    oracle.DAS, oracle.make_rule())
    c0 = r["dcount"]
    pts = c0[0] * c0[1]
    for l in range(1, r["n_logged"]):       # iterations 2.. image the region before them
        lo, hi = r["box_lo"][l - 1], r["box_hi"][l - 1]
        pts += oracle.region_lattice(lo[0], hi[0], c0[0])[2] * \
            oracle.region_lattice(lo[1], hi[1], c0[1])[2]
    pts += (r["roi_hi"][0] - r["roi_lo"][0]) * (r["roi_hi"][1] - r["roi_lo"][1])
    assert r["points_evaluated"] == pts


@pytest.mark.parametrize("bf", [oracle.DAS, oracle.DMAS])
def test_progressive_noiseless_scatterer_at_its_pixel(bf):
    cfg = phantom.with_changes(phantom.CONFIGS["dmas2d_512"], grid_n=(128, 128, 1), extent=0.08,
                               snr_db=None, n_clutter=0)
    g = cfg.grid()
    ants = phantom.antenna_positions(cfg).astype(np.float32)
    for ix, iy in [(41, 87), (100, 20), (64, 63)]:
        p = [g["origin"][0] + ix * g["pitch"][0], g["origin"][1] + iy * g["pitch"][1], 0.0]
        tr = phantom.point_scatterer_traces(cfg, [p], [1.0])
        r = oracle.localize_progressive(tr, ants, g, cfg.v, cfg.fs, cfg.window, bf,
                                        oracle.make_rule())
        assert r["loc_idx"][:2] == [ix, iy]
