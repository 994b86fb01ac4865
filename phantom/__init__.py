"""Seeded synthetic monostatic UWB scans of a breast phantom.

This module only *makes inputs*. It holds none of the imaging method's
arithmetic (no beamforming, no decimation, no segment selection); both the
FP64 oracle and the CUDA path consume what it produces.

Forward model (the paper's own FDTD phantoms, Section IV, are not available, so
these scenes stand in for them):

* antennas: a ring (2-D) or a Fibonacci hemisphere (3-D) of radius ``radius``;
* point scatterers ``s`` (tumours and clutter) with amplitude ``A_s`` and their
  own relative permittivity ``eps_s`` (so their own speed ``v_s = c/sqrt(eps_s)``);
* the monostatic echo at antenna ``a_i`` is
  ``Y_i[n] = sum_s A_s * p(n/fs - 2|r_s - a_i| / v_s) + noise``;
* ``p`` is a differentiated Gaussian with unit peak magnitude,
  ``p(t) = -(t/sigma) * exp(1/2 - t^2 / (2 sigma^2))``, ``sigma = 1/(2 pi f_c)``;
* white Gaussian noise whose power is the mean clean-signal power over the echo
  span divided by ``10^(SNR/10)``.

Every random draw comes from ``numpy.random.Philox`` seeded with
``base_seed + scan_index``, so a scan is reproducible on any machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

C0 = 299_792_458.0
BASE_SEED = 1_709_025_490
_PULSE_HALF_WIDTH_SIGMAS = 12.0  # p(t) < 1e-29 beyond 12 sigma


@dataclasses.dataclass(frozen=True)
class ScanConfig:
    """Geometry, medium, pulse and scene statistics of one workload."""

    name: str
    dim: int                       # 2 or 3
    n_antennas: int
    array: str                     # "ring" | "hemisphere"
    radius: float                  # antenna radius [m]
    grid_n: tuple                  # points per axis (x, y, z); z = 1 in 2-D
    extent: float                  # side of the imaged square / cube [m]
    n_samples: int
    fs: float = 50e9
    window: int = 20
    eps_r: float = 9.0
    f_center: float = 6e9
    snr_db: float | None = 20.0    # None = noiseless
    n_tumors: tuple = (1, 1)       # inclusive range
    tumor_amp: tuple = (1.0, 1.0)
    tumor_half: float = 0.04       # tumours drawn in [-tumor_half, tumor_half]^dim
    antenna_clearance: float = 0.01
    n_clutter: int = 0
    clutter_amp: tuple = (0.05, 0.2)
    eps_jitter: float = 0.0        # clutter eps_s = eps_r * (1 + U[-j, j])
    min_tumor_diameter: float = 0.01

    @property
    def v(self) -> float:
        return C0 / math.sqrt(self.eps_r)

    @property
    def pitch(self) -> float:
        return self.extent / self.grid_n[0]

    def grid(self) -> dict:
        """Lattice of focal points: point ``idx`` sits at ``origin + idx * pitch``
        (cell centres of a cube/square of side ``extent`` centred on 0)."""
        n = list(self.grid_n) + [1] * (3 - len(self.grid_n))
        origin = [-self.extent / 2 + self.pitch / 2 if n[a] > 1 else 0.0 for a in range(3)]
        pitch = [self.pitch if n[a] > 1 else 1.0 for a in range(3)]
        return {"dim": self.dim, "n": n, "origin": origin, "pitch": pitch}


# The three workloads: a 2-D DAS scene, a 2-D DMAS scene with clutter and a 3-D
# hemispherical scene.  Sizes follow the stated benchmark configurations.
CONFIGS = {
    "das2d_64": ScanConfig(
        name="das2d_64", dim=2, n_antennas=16, array="ring", radius=0.06,
        grid_n=(64, 64, 1), extent=0.10, n_samples=1024, snr_db=20.0,
        tumor_half=0.04),
    "dmas2d_512": ScanConfig(
        name="dmas2d_512", dim=2, n_antennas=32, array="ring", radius=0.07,
        grid_n=(512, 512, 1), extent=0.12, n_samples=2048, snr_db=15.0,
        tumor_half=0.05, n_clutter=50, clutter_amp=(0.05, 0.2), eps_jitter=0.10),
    "hemi3d_256": ScanConfig(
        name="hemi3d_256", dim=3, n_antennas=64, array="hemisphere", radius=0.07,
        grid_n=(256, 256, 256), extent=0.10, n_samples=4096, snr_db=15.0,
        n_tumors=(1, 3), tumor_amp=(0.5, 1.0), tumor_half=0.04,
        n_clutter=100, clutter_amp=(0.05, 0.2), eps_jitter=0.10),
}


# Multistatic ring of 12 antennas (the paper's experiments use a ring of 12),
# every transmitter/receiver pair recorded (Eq. 4 sums over all of them).
CONFIGS["ms2d_12"] = ScanConfig(
    name="ms2d_12", dim=2, n_antennas=12, array="ring", radius=0.07, grid_n=(256, 256, 1),
    extent=0.12, n_samples=2048, snr_db=20.0, tumor_half=0.05, n_clutter=20,
    clutter_amp=(0.05, 0.2), eps_jitter=0.10)


def ragged_configs(n_scans: int, seed: int = BASE_SEED, dim: int = 2,
                   max_antennas: int = 96) -> list:
    """Per-scan workloads of a batch of uneven scans: each draws 16-96 antennas
    (16-max_antennas), 1024-4096 samples and a 2-D grid side of 128-1024 points
    (or a 128^3 cube when dim == 3) over a 12 cm region, with the clutter,
    permittivity jitter and 15 dB noise of the 512 x 512 workload."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    base = CONFIGS["dmas2d_512"]
    for _ in range(n_scans):
        m = int(rng.integers(16, max_antennas + 1))
        n = int(rng.integers(1024, 4097))
        if dim == 2:
            g = int(rng.integers(128, 1025))
            out.append(with_changes(base, name="ragged", n_antennas=m, n_samples=n,
                                    grid_n=(g, g, 1)))
        else:
            out.append(with_changes(CONFIGS["hemi3d_256"], name="ragged3d", n_antennas=m,
                                    n_samples=n, grid_n=(128, 128, 128)))
    return out


def all_channels(m: int) -> np.ndarray:
    """[m*m, 2] (transmitter, receiver) pairs, transmitter-major."""
    tx, rx = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    return np.stack([tx.ravel(), rx.ravel()], 1).astype(np.int32)


def with_changes(cfg: ScanConfig, **kw) -> ScanConfig:
    return dataclasses.replace(cfg, **kw)


def antenna_positions(cfg: ScanConfig) -> np.ndarray:
    """[M, 3] antenna centres in metres (float64)."""
    m = cfg.n_antennas
    if cfg.array == "ring":
        ang = 2.0 * np.pi * np.arange(m) / m
        return np.stack([cfg.radius * np.cos(ang), cfg.radius * np.sin(ang),
                         np.zeros(m)], axis=1)
    if cfg.array == "hemisphere":
        golden = np.pi * (3.0 - math.sqrt(5.0))
        z = cfg.radius * (np.arange(m) + 0.5) / m
        rho = np.sqrt(cfg.radius ** 2 - z ** 2)
        phi = golden * np.arange(m)
        return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    raise ValueError(f"unknown array {cfg.array!r}")


def pulse(t: np.ndarray, sigma: float) -> np.ndarray:
    """Differentiated Gaussian with unit peak magnitude (peaks at t = -/+ sigma)."""
    x = t / sigma
    return -x * np.exp(0.5 - 0.5 * x * x)


def _inside(cfg: ScanConfig, p: np.ndarray) -> bool:
    if np.linalg.norm(p) > cfg.radius - cfg.antenna_clearance:
        return False
    if cfg.dim == 3 and p[2] < 0.0:
        return False
    return True


def _draw_point(cfg, rng, half, ants):
    for _ in range(10_000):
        p = np.zeros(3)
        p[:cfg.dim] = rng.uniform(-half, half, size=cfg.dim)
        if cfg.dim == 3:
            p[2] = abs(p[2])
        if not _inside(cfg, p):
            continue
        if np.min(np.linalg.norm(ants - p, axis=1)) < cfg.antenna_clearance:
            continue
        return p
    raise RuntimeError("could not place a scatterer")


def draw_scene(cfg: ScanConfig, seed: int) -> dict:
    """Scatterer list and noise stream for one scan (all from one Philox stream)."""
    rng = np.random.Generator(np.random.Philox(seed))
    ants = antenna_positions(cfg)
    nt = int(rng.integers(cfg.n_tumors[0], cfg.n_tumors[1] + 1))
    pos, amp, eps = [], [], []
    for _ in range(nt):
        pos.append(_draw_point(cfg, rng, cfg.tumor_half, ants))
        amp.append(rng.uniform(*cfg.tumor_amp) if cfg.tumor_amp[0] != cfg.tumor_amp[1]
                   else cfg.tumor_amp[0])
        eps.append(cfg.eps_r)
    half_region = cfg.extent / 2
    for _ in range(cfg.n_clutter):
        pos.append(_draw_point(cfg, rng, half_region, ants))
        amp.append(rng.uniform(*cfg.clutter_amp))
        eps.append(cfg.eps_r * (1.0 + rng.uniform(-cfg.eps_jitter, cfg.eps_jitter))
                   if cfg.eps_jitter > 0 else cfg.eps_r)
    return {"rng": rng, "antennas": ants, "pos": np.array(pos), "amp": np.array(amp),
            "eps": np.array(eps), "n_tumors": nt}


def echo_span(cfg: ScanConfig) -> int:
    """Samples covering every round trip from an antenna to the imaged box and
    back at the slowest scatterer speed (used only to define the noise power)."""
    ants = antenna_positions(cfg)
    g = cfg.grid()
    corners = []
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                c = [g["origin"][a] + (g["n"][a] - 1) * g["pitch"][a] * (cx, cy, cz)[a]
                     for a in range(3)]
                corners.append(c)
    dmax = max(np.linalg.norm(ants - np.array(c), axis=1).max() for c in corners)
    vmin = C0 / math.sqrt(cfg.eps_r * (1.0 + cfg.eps_jitter))
    return min(cfg.n_samples, int(math.ceil(2.0 * dmax / vmin * cfg.fs)) + cfg.window + 2)


def synthesize(cfg: ScanConfig, pos, amp, eps, ants, channels=None) -> np.ndarray:
    """Clean traces (float64) for a list of point scatterers: [M, N] monostatic
    echoes, or [C, N] for channels [C, 2] = (transmitter, receiver) pairs, whose
    round trip is |r_s - a_tx| + |r_s - a_rx| at the scatterer's speed."""
    n = cfg.n_samples
    m = cfg.n_antennas if channels is None else len(channels)
    sigma = 1.0 / (2.0 * np.pi * cfg.f_center)
    half = int(math.ceil(_PULSE_HALF_WIDTH_SIGMAS * sigma * cfg.fs)) + 1
    out = np.zeros(m * n)
    if len(pos) == 0:
        return out.reshape(m, n)
    vs = C0 / np.sqrt(np.asarray(eps))                                  # [S]
    dist = np.linalg.norm(pos[:, None, :] - ants[None, :, :], axis=2)   # [S, M]
    if channels is None:
        path = 2.0 * dist
    else:
        ch = np.asarray(channels)
        path = dist[:, ch[:, 0]] + dist[:, ch[:, 1]]                    # [S, C]
    tau = path / vs[:, None]                                            # seconds
    centre = np.floor(tau * cfg.fs).astype(np.int64)
    offs = np.arange(-half, half + 1)
    idx = centre[:, :, None] + offs[None, None, :]                      # [S, M, K]
    t = idx / cfg.fs - tau[:, :, None]
    val = np.asarray(amp)[:, None, None] * pulse(t, sigma)
    ok = (idx >= 0) & (idx < n)
    flat = (np.arange(m)[None, :, None] * n + idx)[ok]
    out += np.bincount(flat, weights=val[ok], minlength=m * n)
    return out.reshape(m, n)


def make_scan(cfg: ScanConfig, seed: int, channels=None) -> dict:
    """One scan: float32 traces [M, N] (or [C, N] for multistatic channels),
    float32 antennas [M, 3] and the truth."""
    sc = draw_scene(cfg, seed)
    clean = synthesize(cfg, sc["pos"], sc["amp"], sc["eps"], sc["antennas"], channels)
    traces = clean
    if cfg.snr_db is not None:
        span = echo_span(cfg)
        p_sig = float(np.mean(clean[:, :span] ** 2))
        sigma_n = math.sqrt(p_sig / 10.0 ** (cfg.snr_db / 10.0))
        traces = clean + sigma_n * sc["rng"].standard_normal(clean.shape)
    nt = sc["n_tumors"]
    return {
        "traces": traces.astype(np.float32),
        "antennas": sc["antennas"].astype(np.float32),
        "tumors": sc["pos"][:nt].copy(),
        "tumor_amp": sc["amp"][:nt].copy(),
        "scatterers": sc["pos"].copy(),
        "channels": None if channels is None else np.asarray(channels, np.int32),
    }


def make_batch(cfg: ScanConfig, n_scans: int, first_scan: int = 0,
               base_seed: int = BASE_SEED, channels=None) -> dict:
    """``n_scans`` scans with seeds ``base_seed + first_scan + s``.

    Returns traces float32 [B, M, N] ([B, C, N] with channels), antennas
    float32 [M, 3] (one array geometry per workload) and per-scan tumour lists.
    """
    rows = cfg.n_antennas if channels is None else len(channels)
    tr = np.empty((n_scans, rows, cfg.n_samples), dtype=np.float32)
    tumors = []
    ants = None
    for s in range(n_scans):
        sc = make_scan(cfg, base_seed + first_scan + s, channels)
        tr[s] = sc["traces"]
        ants = sc["antennas"]
        tumors.append(sc["tumors"])
    return {"traces": tr, "antennas": ants, "tumors": tumors, "grid": cfg.grid(),
            "v": cfg.v, "fs": cfg.fs, "window": cfg.window,
            "channels": None if channels is None else np.asarray(channels, np.int32)}


def point_scatterer_traces(cfg: ScanConfig, points: Sequence, amps: Sequence,
                           ants: np.ndarray | None = None) -> np.ndarray:
    """Noiseless float32 traces of point scatterers in the nominal medium."""
    if ants is None:
        ants = antenna_positions(cfg)
    pos = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    eps = np.full(len(pos), cfg.eps_r)
    return synthesize(cfg, pos, np.asarray(amps, dtype=np.float64), eps, ants).astype(np.float32)
