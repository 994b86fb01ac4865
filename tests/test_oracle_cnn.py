"""Pins of the FP64 oracle of the learned segment proposal (oracle/cnn.py).

Each pin checks the oracle against something other than itself: SciPy's
correlation, finite differences, closed forms, torch's bfloat16 conversion and
a network built by hand whose output is known in closed form.
"""
import numpy as np
import pytest

import phantom
import oracle
from oracle import cnn

scipy_signal = pytest.importorskip("scipy.signal")


def _rng(seed):
    return np.random.Generator(np.random.Philox(seed))


def _hand_network(gain: float, tap: int = 4) -> np.ndarray:
    """Channel 0 carries the normalised map through all three layers (tap
    `tap` of layer 1, centre taps after it); every other weight is zero. The
    scores are then gain x the segment means of the (rounded) map."""
    P = cnn.unpack(np.zeros(cnn.N_PARAMS))
    P["W1"][0, tap] = 1.0
    P["W2"][0, 4, 0] = 1.0
    P["W3"][0, 4, 0] = 1.0
    P["wh"][0] = gain
    return cnn.pack(P)


# ------------------------------------------------------------------ arithmetic pins

def test_bf16_rounding_hand_values():
    one = 1.0
    assert cnn.bf16(np.array([one]))[0] == 1.0
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    assert cnn.bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert cnn.bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6
    assert cnn.bf16(np.array([-(1 + 2.0 ** -7 + 2.0 ** -9)]))[0] == -(1 + 2.0 ** -7)
    assert cnn.bf16(np.array([0.0]))[0] == 0.0


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = _rng(3).normal(0, 10, 20000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.bf16(x), ref)


def test_conv_matches_scipy_correlation():
    rng = _rng(5)
    X = rng.normal(size=(2, 3, 32, 32))
    W = rng.normal(size=(4, 9, 3))
    Z = cnn.conv(X, W)
    for b in range(2):
        for o in range(4):
            ref = np.zeros((32, 32))
            for c in range(3):
                K = W[o, :, c].reshape(3, 3)          # K[dy + 1, dx + 1]
                ref += scipy_signal.correlate2d(X[b, c], K, mode="same", boundary="fill")
            np.testing.assert_allclose(Z[b, o], ref, rtol=1e-12, atol=1e-12)


def test_tap_convention_shifts_the_map():
    # tap 5 is (dy, dx) = (0, +1): channel 0 of layer 1 reads the right neighbour
    rng = _rng(7)
    E = rng.uniform(0.1, 1.0, (1, 32, 32))
    f = cnn.forward(_hand_network(1.0, tap=5), E, quantise=False)
    X0 = E[0] / E.max()
    want = np.zeros_like(X0)
    want[:, :-1] = X0[:, 1:]
    np.testing.assert_allclose(f["A1"][0, 0], want, rtol=1e-15)


def test_hand_network_scores_are_segment_means():
    rng = _rng(11)
    E = rng.uniform(0.0, 1.0, (3, 32, 32))
    gain = 7.5
    f = cnn.forward(_hand_network(gain), E)
    X0 = cnn.bf16(E / E.reshape(3, -1).max(1)[:, None, None])
    means = X0.reshape(3, 4, 8, 4, 8).mean(axis=(2, 4)).reshape(3, 16)
    np.testing.assert_allclose(f["z"], gain * means, rtol=1e-14)
    np.testing.assert_allclose(f["p"].sum(1), 1.0, rtol=1e-14)


def test_zero_network_is_uniform_with_loss_log16():
    theta = np.zeros(cnn.N_PARAMS)
    E = _rng(13).uniform(0, 1, (5, 32, 32))
    labels = np.arange(5)
    loss, g = cnn.loss_and_grad(theta, E, labels)
    assert loss == pytest.approx(np.log(16.0), rel=1e-14)
    f = cnn.forward(theta, E)
    np.testing.assert_allclose(f["p"], 1.0 / 16.0)
    # all activations are zero, so only the head bias sees a gradient, and the
    # softmax gradient sums to zero over the segments (up to rounding)
    assert np.all(g[:-1] == 0.0)
    assert abs(g[-1]) < 1e-15


def test_gradient_matches_finite_differences():
    rng = _rng(17)
    theta = cnn.init_params(99).astype(np.float64)
    theta[cnn.N_PARAMS - 33:] *= 3.0                 # a livelier head
    P = cnn.unpack(theta)
    for name in ("b1", "b2", "b3"):
        P[name] = rng.uniform(0.0, 0.1, P[name].shape)
    theta = cnn.pack(P)
    E = rng.uniform(0.0, 1.0, (3, 32, 32))
    labels = np.array([2, 9, 15])
    loss, g = cnn.loss_and_grad(theta, E, labels, quantise=False)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in cnn.SIZES])
    idx = np.concatenate([rng.choice(np.arange(offs[k], offs[k + 1]),
                                     size=min(8, offs[k + 1] - offs[k]), replace=False)
                          for k in range(len(cnn.SIZES))])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (cnn.loss_and_grad(tp, E, labels, quantise=False)[0]
              - cnn.loss_and_grad(tm, E, labels, quantise=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_adam_first_step_is_a_signed_lr_step():
    rng = _rng(19)
    theta = rng.normal(size=50)
    grad = rng.normal(size=50)
    new, m, v = cnn.adam_step(theta, np.zeros(50), np.zeros(50), grad, 1, lr=1e-3)
    # m_hat = g and v_hat = g^2 after one step
    np.testing.assert_allclose(new, theta - 1e-3 * grad / (np.abs(grad) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * grad, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * grad * grad, rtol=1e-14)


def test_pack_unpack_round_trip_and_count():
    assert cnn.N_PARAMS == 32 * 9 + 32 + 2 * (32 * 9 * 32 + 32) + 32 + 1
    theta = np.arange(cnn.N_PARAMS, dtype=np.float64)
    np.testing.assert_array_equal(cnn.pack(cnn.unpack(theta)), theta)


# ------------------------------------------------------------ learned localisation

def _cfg128():
    return phantom.with_changes(phantom.CONFIGS["dmas2d_512"], grid_n=(128, 128, 1),
                                extent=0.08, snr_db=None, n_clutter=0)


def test_map_lattice_and_segments():
    l0, st, ct = cnn.map_lattice((0, 0), 512)
    assert (l0, st, ct) == ([7, 7, 0], [16, 16, 1], [32, 32, 1])
    l0, st, ct = cnn.map_lattice((128, 256), 128)
    assert (l0, st, ct) == ([129, 257, 0], [4, 4, 1], [32, 32, 1])
    assert cnn.segment_box((0, 0), 512, 6) == ((256, 128), 128)
    assert cnn.segment_box((128, 256), 128, 15) == ((224, 352), 32)


def test_hand_network_localises_a_noiseless_scatterer_at_its_pixel():
    cfg = _cfg128()
    g = cfg.grid()
    ants = phantom.antenna_positions(cfg).astype(np.float32)
    theta = _hand_network(200.0)
    rule = oracle.make_rule()
    for ix, iy in [(41, 87), (100, 20), (70, 70)]:
        p = [g["origin"][0] + ix * g["pitch"][0], g["origin"][1] + iy * g["pitch"][1], 0.0]
        tr = phantom.point_scatterer_traces(cfg, [p], [1.0])
        for bf in (oracle.DAS, oracle.DMAS):
            r = cnn.learned_localize(tr, ants, g, cfg.v, cfg.fs, cfg.window, theta, 0.5, bf,
                                     rule, localize=oracle.localize, image=oracle.image)
            assert not r["fallback"]
            assert r["loc_idx"] == [ix, iy]
            # the proposed segments contain the scatterer
            assert r["segments"][0] == 4 * (iy // 32) + ix // 32
            assert r["segments"][1] == 4 * ((iy % 32) // 8) + (ix % 32) // 8


def test_below_threshold_the_plain_framework_decides():
    cfg = _cfg128()
    g = cfg.grid()
    ants = phantom.antenna_positions(cfg).astype(np.float32)
    p = [0.011, -0.017, 0.0]
    tr = phantom.point_scatterer_traces(cfg, [p], [1.0])
    rule = oracle.make_rule()
    r = cnn.learned_localize(tr, ants, g, cfg.v, cfg.fs, cfg.window, _hand_network(200.0), 1.01,
                             oracle.DAS, rule, localize=oracle.localize, image=oracle.image)
    assert r["fallback"]
    ref = oracle.localize(tr, ants, g, cfg.v, cfg.fs, cfg.window, oracle.DAS, rule)
    assert r["loc_idx"] == ref["loc_idx"][:2]


def test_shipped_weights_load_with_their_training_record():
    from paper_1709_02549_gb300 import proposal
    theta, record = proposal.load()
    assert theta.shape == (cnn.N_PARAMS,) and theta.dtype == np.float32
    assert np.all(np.isfinite(theta))
    assert record["workload"] == "dmas2d_512"
    assert record["train_scans"] >= 100_000
    assert 0.0 < record["threshold"] <= 1.0
    # training, validation and evaluation seeds never overlap the benchmark's
    assert record["train_first_scan"] >= 1_000_000
    # the proposal's own initialisation follows the oracle's parameter layout
    assert proposal.N_PARAMS == cnn.N_PARAMS
    assert [tuple(s) for s in proposal.SIZES] == [s for _, s in cnn.SIZES]
