"""The synthetic scan generator: pulse shape, echo timing and seeding."""
import math

import numpy as np
import pytest

import phantom


def test_pulse_is_a_unit_peak_differentiated_gaussian():
    sigma = 1.0 / (2 * math.pi * 6e9)
    t = np.linspace(-6 * sigma, 6 * sigma, 20001)
    p = phantom.pulse(t, sigma)
    assert np.max(np.abs(p)) == pytest.approx(1.0, rel=1e-6)
    assert t[np.argmax(p)] == pytest.approx(-sigma, rel=1e-3)
    assert t[np.argmin(p)] == pytest.approx(sigma, rel=1e-3)
    np.testing.assert_allclose(p, -p[::-1], atol=1e-12)       # odd


def test_noiseless_echo_crosses_zero_at_the_round_trip_delay():
    cfg = phantom.with_changes(phantom.CONFIGS["das2d_64"], snr_db=None)
    ants = phantom.antenna_positions(cfg)
    p = np.array([0.013, -0.021, 0.0])
    tr = phantom.point_scatterer_traces(cfg, [p], [1.0], ants).astype(np.float64)
    for i in range(cfg.n_antennas):
        u = 2 * np.linalg.norm(p - ants[i]) / cfg.v * cfg.fs
        n0 = int(math.floor(u))
        # the odd pulse changes sign across its centre u
        assert tr[i, n0 - 1] > 0 > tr[i, n0 + 2]
        assert abs(np.argmax(np.abs(tr[i])) - u) < 3.0


def test_scans_are_reproducible_and_distinct():
    cfg = phantom.CONFIGS["das2d_64"]
    a = phantom.make_scan(cfg, phantom.BASE_SEED + 5)
    b = phantom.make_scan(cfg, phantom.BASE_SEED + 5)
    c = phantom.make_scan(cfg, phantom.BASE_SEED + 6)
    np.testing.assert_array_equal(a["traces"], b["traces"])
    assert not np.array_equal(a["traces"], c["traces"])


def test_snr_sets_the_noise_power():
    cfg = phantom.CONFIGS["dmas2d_512"]
    sc = phantom.make_scan(cfg, phantom.BASE_SEED)
    clean_cfg = phantom.with_changes(cfg, snr_db=None)
    clean = phantom.make_scan(clean_cfg, phantom.BASE_SEED)["traces"].astype(np.float64)
    noise = sc["traces"].astype(np.float64) - clean
    span = phantom.echo_span(cfg)
    snr = 10 * math.log10(np.mean(clean[:, :span] ** 2) / np.mean(noise ** 2))
    assert snr == pytest.approx(cfg.snr_db, abs=0.3)


def test_tumours_stay_inside_the_array():
    for name, cfg in phantom.CONFIGS.items():
        for s in range(3):
            sc = phantom.make_scan(cfg, phantom.BASE_SEED + s)
            for t in sc["tumors"]:
                assert np.linalg.norm(t) <= cfg.radius - cfg.antenna_clearance + 1e-12
                assert np.all(np.abs(t[:cfg.dim]) <= cfg.extent / 2)
