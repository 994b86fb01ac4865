"""The learned segment proposal on the GPU against its FP64 oracle
(oracle/cnn.py), through the C ABI (needs a GB300).

Comparison. The kernels write a record of every intermediate of the forward
pass (uwb_cnn_forward_record; the gradient call overwrites two of its slots
with the backward pass's BF16 pre-activation gradients). Each step is then
recomputed by the oracle from the kernels' own stored inputs of that step and
compared element by element, within bounds derived from where the kernels
round (oracle/cnn_check.py): FP32 accumulation of K terms, at most
K * 2^-23 * sum |term|, plus one BF16 step where the result is stored in
BF16. Decisions (the proposed segment) must equal the oracle's where the
oracle's own score margin is clear.
"""
import numpy as np
import pytest
import torch

import oracle
import phantom
from oracle import cnn, cnn_check
from parity import dev, record_to_dict

pytestmark = pytest.mark.gpu

# the proposed segment must be the oracle's where the oracle's two best
# scores differ by more than this fraction of the largest score magnitude
CLEAR_MARGIN = 4e-2


def _rng(seed):
    return np.random.Generator(np.random.Philox(seed))


def random_theta(seed, bias=0.05):
    rng = _rng(seed)
    P = cnn.unpack(cnn.init_params(seed).astype(np.float64))
    for name in ("b1", "b2", "b3"):
        P[name] = rng.uniform(-bias, bias, 32)
    P["wh"] *= 4.0
    P["bh"] = np.array([0.3])
    return cnn.pack(P).astype(np.float32)


def random_maps(seed, B):
    """Coarse-energy-like maps: a positive background with a few blobs, one
    all-zero map and one single spike."""
    rng = _rng(seed)
    y, x = np.mgrid[0:32, 0:32]
    maps = rng.gamma(2.0, 0.05, (B, 32, 32))
    for b in range(B):
        for _ in range(rng.integers(1, 4)):
            cy, cx = rng.uniform(0, 32, 2)
            w = rng.uniform(1.0, 3.0)
            maps[b] += rng.uniform(0.5, 3.0) * np.exp(-((y - cy) ** 2 + (x - cx) ** 2) / (2 * w * w))
    if B > 2:
        maps[1] = 0.0
        maps[2] = 0.0
        maps[2, 17, 3] = 5.0
    return (maps * 1e3).astype(np.float32)   # raw energies: scale is normalised away


def packed_of(gpu, theta):
    th = dev(theta)
    pk = torch.zeros(gpu.CNN_PACKED_BYTES, dtype=torch.uint8, device="cuda")
    gpu.uwb_cnn_pack(th, pk)
    return th, pk


def test_tensor_core_selfcheck_passes(gpu):
    assert gpu.uwb_cnn_selftest()


def test_packed_weights_are_the_bf16_rounding(gpu):
    theta = random_theta(3)
    _, pk = packed_of(gpu, theta)
    torch.cuda.synchronize()
    raw = pk.cpu().numpy()
    w2 = raw[1024:1024 + 2 * 9216].view(np.uint16).astype(np.uint32) << 16
    P = cnn.unpack(theta.astype(np.float64))
    np.testing.assert_array_equal(w2.view(np.float32).astype(np.float64),
                                  cnn.bf16(P["W2"]).ravel())
    f32 = raw[37888:37888 + 129 * 4].view(np.float32)
    np.testing.assert_array_equal(f32[:32], P["b1"].astype(np.float32))
    np.testing.assert_array_equal(f32[96:128], P["wh"].astype(np.float32))
    assert f32[128] == np.float32(P["bh"][0])


def forward_record(gpu, pk, maps, labels=None):
    B = maps.shape[0]
    scores = torch.full((B, 16), float("nan"), device="cuda")
    rec = torch.empty(B * gpu.CNN_RECORD_BYTES, dtype=torch.uint8, device="cuda")
    loss = torch.zeros(1, device="cuda") if labels is not None else None
    gpu.uwb_cnn_forward_record(pk, dev(maps), scores, rec,
                               None if labels is None else dev(labels, torch.int32), loss)
    torch.cuda.synchronize()
    return scores.cpu().numpy().astype(np.float64), rec, loss


@pytest.mark.parametrize("B", [1, 7, 300])
def test_forward_matches_oracle_layer_by_layer(gpu, B):
    theta = random_theta(11)
    maps = random_maps(100 + B, B)
    _, pk = packed_of(gpu, theta)
    got, rec, _ = forward_record(gpu, pk, maps)
    plain = torch.full((B, 16), float("nan"), device="cuda")
    gpu.uwb_cnn_forward(pk, dev(maps), plain)
    torch.cuda.synchronize()
    # writing the record changes no score
    np.testing.assert_array_equal(plain.cpu().numpy().astype(np.float64), got)
    idx = np.arange(B) if B <= 16 else np.sort(_rng(5).choice(B, 16, replace=False))
    arr = gpu.cnn_record_arrays(rec.cpu().numpy(), B)
    cnn_check.check_forward(theta, maps[idx], {k: v[idx] for k, v in arr.items()}, got[idx])
    # the proposed segment is the oracle's wherever the oracle's margin is clear
    ref = cnn.forward(theta, maps[idx])["z"]
    scale = np.abs(ref).max(axis=1) + 1e-3
    zs = np.sort(ref, axis=1)
    clear = (zs[:, -1] - zs[:, -2]) > CLEAR_MARGIN * scale
    np.testing.assert_array_equal(np.argmax(got[idx], 1)[clear], np.argmax(ref, 1)[clear])


def test_gradients_match_oracle_step_by_step(gpu):
    B = 6
    theta = random_theta(21)
    maps = random_maps(7, B)
    labels = np.array([3, 0, 15, 7, 7, 12], np.int32)
    _, pk = packed_of(gpu, theta)
    scores, rec, _ = forward_record(gpu, pk, maps, labels)
    grad = torch.full((gpu.CNN_PARAMS,), float("nan"), device="cuda")
    loss = torch.zeros(1, device="cuda")
    ws = torch.empty(gpu.uwb_cnn_train_workspace(B), dtype=torch.uint8, device="cuda")
    gpu.uwb_cnn_gradients(pk, dev(maps), dev(labels, torch.int32), grad, loss, ws)
    torch.cuda.synchronize()
    fwd = gpu.cnn_record_arrays(rec.cpu().numpy(), B)
    bwd = gpu.cnn_record_arrays(ws[:B * gpu.CNN_RECORD_BYTES].cpu().numpy(), B)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(g))
    cnn_check.check_forward(theta, maps, fwd, scores)
    cnn_check.check_backward(theta, labels, fwd, bwd, scores, g, float(loss.item()))


def test_adam_matches_oracle(gpu):
    rng = _rng(31)
    n = gpu.CNN_PARAMS
    theta = rng.normal(0, 0.1, n).astype(np.float32)
    m = rng.normal(0, 1e-3, n).astype(np.float32)
    v = rng.uniform(0, 1e-5, n).astype(np.float32)
    g = rng.normal(0, 1e-2, n).astype(np.float32)
    th, mm, vv, gg = dev(theta), dev(m), dev(v), dev(g)
    pk = torch.zeros(gpu.CNN_PACKED_BYTES, dtype=torch.uint8, device="cuda")
    gpu.uwb_cnn_adam(th, mm, vv, gg, pk, 5, 2e-3)
    torch.cuda.synchronize()
    ref, rm, rv = cnn.adam_step(theta, m, v, g.astype(np.float64), 5, 2e-3)
    np.testing.assert_allclose(th.cpu().numpy(), ref, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(mm.cpu().numpy(), rm, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(vv.cpu().numpy(), rv, rtol=1e-5, atol=1e-12)
    assert torch.count_nonzero(gg).item() == 0      # the gradient is consumed
    # and the packed copy follows the new parameters
    sc_pack = torch.zeros_like(pk)
    gpu.uwb_cnn_pack(th, sc_pack)
    torch.cuda.synchronize()
    assert torch.equal(sc_pack, pk)


def test_training_reduces_the_loss(gpu):
    """A few hundred Adam steps on blob maps labelled by the blob's segment."""
    rng = _rng(41)
    B = 128
    y, x = np.mgrid[0:32, 0:32]

    def batch():
        cy, cx = rng.uniform(1, 31, (2, B))
        maps = rng.gamma(2.0, 0.05, (B, 32, 32))
        maps += np.exp(-((y[None] - cy[:, None, None]) ** 2 +
                         (x[None] - cx[:, None, None]) ** 2) / 2.0)
        lab = (4 * (cy // 8) + cx // 8).astype(np.int32)
        return dev(maps.astype(np.float32)), dev(lab, torch.int32)

    th = dev(cnn.init_params(5))
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    pk = torch.zeros(gpu.CNN_PACKED_BYTES, dtype=torch.uint8, device="cuda")
    gpu.uwb_cnn_pack(th, pk)
    ws = torch.empty(gpu.uwb_cnn_train_workspace(B), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(1, device="cuda")
    first = []
    last = []
    for step in range(1, 301):
        mp, lb = batch()
        gpu.uwb_cnn_train_step(th, m, v, pk, mp, lb, step, 2e-3, loss, ws)
        if step <= 5:
            first.append(loss.item())
        if step > 290:
            last.append(loss.item())
    assert np.mean(first) > 2.0
    assert np.mean(last) < 0.6 * np.mean(first)
    mp, lb = batch()
    scores = torch.empty(B, 16, device="cuda")
    gpu.uwb_cnn_forward(pk, mp, scores)
    acc = (scores.argmax(1).int() == lb).float().mean().item()
    assert acc > 0.7, acc


# ------------------------------------------------------------------ coarse maps

def _scan_batch(cfg, B, first):
    b = phantom.make_batch(cfg, B, first)
    return b["traces"], b["antennas"].astype(np.float32), b["grid"], b["v"], b["fs"], b["window"]


def test_coarse_maps_match_oracle(gpu):
    cfg = phantom.CONFIGS["dmas2d_512"]
    tr, ants, g, v, fs, W = _scan_batch(cfg, 3, 900)
    B = tr.shape[0]
    maps = torch.full((B, 32, 32), -1.0, device="cuda")
    gpu.uwb_coarse_maps(dev(tr), dev(ants), g, v, fs, W, 512, maps)
    lo = np.array([[128, 256], [0, 384], [384, 0]], np.int32)
    maps2 = torch.full((B, 32, 32), -1.0, device="cuda")
    ws = torch.empty(gpu.uwb_coarse_maps_workspace(B), dtype=torch.uint8, device="cuda")
    gpu.uwb_coarse_maps(dev(tr), dev(ants), g, v, fs, W, 128, maps2, dev(lo, torch.int32), ws)
    torch.cuda.synchronize()
    for b in range(B):
        for m, (l0, st, ct) in ((maps, cnn.map_lattice((0, 0), 512)),
                                (maps2, cnn.map_lattice(tuple(lo[b]), 128))):
            ref = oracle.image(tr[b], ants, g, v, fs, W, oracle.DAS, lo=l0, step=st, cnt=ct)[0]
            got = m[b].cpu().numpy()
            assert np.abs(got - ref).max() <= 1e-4 * ref.max()


# ------------------------------------------------------------ learned localisation

def _hand_theta(gain):
    P = cnn.unpack(np.zeros(cnn.N_PARAMS))
    P["W1"][0, 4] = 1.0
    P["W2"][0, 4, 0] = 1.0
    P["W3"][0, 4, 0] = 1.0
    P["wh"][0] = gain
    return cnn.pack(P).astype(np.float32)


def gpu_learned(gpu, tr, ants, g, v, fs, W, bf, rule, theta, threshold, levels=2):
    B = tr.shape[0]
    _, pk = packed_of(gpu, theta)
    ws = torch.empty(gpu.uwb_localize_learned_workspace(B, g, rule), dtype=torch.uint8,
                     device="cuda")
    out = torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    gpu.uwb_localize_learned(dev(tr), dev(ants), g, v, fs, W, bf, rule, pk, threshold, levels, ws,
                             out)
    torch.cuda.synchronize()
    return [record_to_dict(r) for r in gpu.results_from_device(out)]


def _orc_rule():
    return oracle.make_rule()


@pytest.mark.parametrize("bf", [0, 2])
def test_hand_network_localisation_matches_oracle(gpu, bf):
    cfg = phantom.with_changes(phantom.CONFIGS["dmas2d_512"], grid_n=(128, 128, 1), extent=0.08,
                               snr_db=None, n_clutter=0)
    g = cfg.grid()
    ants = phantom.antenna_positions(cfg).astype(np.float32)
    pts = [(41, 87), (100, 20), (70, 70), (3, 124)]
    tr = np.stack([phantom.point_scatterer_traces(
        cfg, [[g["origin"][0] + ix * g["pitch"][0], g["origin"][1] + iy * g["pitch"][1], 0.0]],
        [1.0]) for ix, iy in pts])
    theta = _hand_theta(200.0)
    res = gpu_learned(gpu, tr, ants, g, cfg.v, cfg.fs, cfg.window, bf, gpu.uwb_default_rule(),
                      theta, 0.5)
    for b, (ix, iy) in enumerate(pts):
        ref = cnn.learned_localize(tr[b], ants, g, cfg.v, cfg.fs, cfg.window, theta, 0.5,
                                   oracle.DAS if bf == 0 else oracle.DMAS, _orc_rule(),
                                   localize=oracle.localize, image=oracle.image)
        r = res[b]
        assert not ref["fallback"]
        assert r["stop_reason"] == gpu.UWB_STOP_LEARNED and r["status"] == 0
        assert r["child"] == ref["segments"]
        assert r["loc_idx"][:2] == ref["loc_idx"] == [ix, iy]
        assert r["roi_lo"][:2] == ref["box_lo"] and r["roi_hi"][:2] == ref["box_hi"]
        assert r["points_evaluated"] == 2 * 1024 + \
            (ref["box_hi"][0] - ref["box_lo"][0]) * (ref["box_hi"][1] - ref["box_lo"][1])


def test_unconfident_scans_fall_back_to_the_framework(gpu):
    """A network with equal scores (confidence 1/16) hands every scan to the
    Eq. 5 framework: same result records as uwb_localize_batch."""
    from parity import gpu_localize_batch
    cfg = phantom.CONFIGS["dmas2d_512"]
    tr, ants, g, v, fs, W = _scan_batch(cfg, 5, 950)
    rule = gpu.uwb_default_rule()
    theta = np.zeros(cnn.N_PARAMS, np.float32)
    res = gpu_learned(gpu, tr, ants, g, v, fs, W, 1, rule, theta, 0.5)
    plain = gpu_localize_batch(gpu, 1, tr, ants, g, v, fs, W, rule)
    for r, p in zip(res, plain):
        assert r["stop_reason"] != gpu.UWB_STOP_LEARNED
        for key in ("status", "iters", "stop_reason", "roi_lo", "roi_hi", "loc_idx", "child",
                    "box_lo", "box_hi"):
            assert r[key] == p[key], key
        assert r["points_evaluated"] == p["points_evaluated"] + 1024


# ------------------------------------------------------------ the trained network

def test_trained_network_gains_over_the_framework(gpu):
    """The shipped weights on held-out scans of the 512 x 512 workload: the same
    locations as the plain Eq. 5 framework (same literal-DMAS final imaging)
    at the same localisation error, from far fewer focal points and in less
    device time."""
    from paper_1709_02549_gb300 import proposal
    theta, record = proposal.load()
    wl = proposal.Workload("dmas2d_512")
    _, pk = packed_of(gpu, theta)
    B = 512
    b = phantom.make_batch(wl.cfg, B, proposal.EVAL_FIRST_SCAN + 50_000)
    tr = dev(b["traces"])
    th = record["threshold"]
    rl = wl.learned(tr, pk, th, gpu.UWB_DMAS_LITERAL)
    rf = wl.framework(tr, gpu.UWB_DMAS_LITERAL)
    agree = np.mean(np.all(rl["loc_idx"][:, :2] == rf["loc_idx"][:, :2], axis=1))
    fallback = np.mean(rl["stop_reason"] != gpu.UWB_STOP_LEARNED)
    g = wl.grid
    truth = np.array([t[0][:2] for t in b["tumors"]])

    def err(r):
        xy = np.stack([g["origin"][a] + r["loc_idx"][:, a] * g["pitch"][a] for a in range(2)], 1)
        return np.mean(np.linalg.norm(xy - truth, axis=1)) * 1e3

    assert agree >= 0.99, agree
    assert fallback <= 0.05, fallback
    assert rl["points_evaluated"].mean() <= 0.3 * rf["points_evaluated"].mean()
    assert err(rl) <= err(rf) + 0.02
    # device time of the two searches on the same scans
    stream = torch.cuda.current_stream()

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_l = timed(lambda: wl.learned(tr, pk, th, gpu.UWB_DMAS_LITERAL))
    t_f = timed(lambda: wl.framework(tr, gpu.UWB_DMAS_LITERAL))
    assert t_l * 2.0 < t_f, (t_l, t_f)


def test_learned_localisation_replays_in_a_cuda_graph(gpu):
    from paper_1709_02549_gb300 import proposal
    theta, record = proposal.load()
    wl = proposal.Workload("dmas2d_512")
    _, pk = packed_of(gpu, theta)
    b = phantom.make_batch(wl.cfg, 6, proposal.EVAL_FIRST_SCAN + 90_000)
    tr = dev(b["traces"])
    B = tr.shape[0]
    ws = torch.empty(gpu.uwb_localize_learned_workspace(B, wl.grid, wl.rule), dtype=torch.uint8,
                     device="cuda")
    direct = torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")

    def run(out, stream=None):
        gpu.uwb_localize_learned(tr, wl.ants, wl.grid, wl.cfg.v, wl.cfg.fs, wl.cfg.window,
                                 gpu.UWB_DMAS_LITERAL, wl.rule, pk, record["threshold"], 2, ws,
                                 out, stream)

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
