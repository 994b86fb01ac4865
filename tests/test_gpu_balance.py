"""The image kernel's dynamic tile split against its static split and the
oracle (needs a GB300).

With a tile counter the persistent CTAs take chunks of tiles as they free up;
without one each CTA takes an equal contiguous range. The image entry points
take their counter from a per-device pool, so under stream capture (or with
every counter busy) they split statically; the localisation entry points own
their counters in the workspace, zeroed by the call itself, so a graph replay
splits dynamically too. Only the order in which tiles are evaluated differs,
so images, argmaxes and localisations must be byte-identical. The launches
here have at least 16 tiles per CTA (the kernel splits dynamically from 4)
and run several CTAs per SM."""
import numpy as np
import pytest
import torch

import oracle
import phantom
from parity import BF_ORACLE, IMG_TOL, dev, rule_pair

pytestmark = pytest.mark.gpu


def _captured(fn, replays=1):
    """fn(stream) captured into a CUDA graph and replayed: while a stream is
    captured the library takes no counter from its pool, so the image entry
    points split their tiles statically there."""
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        fn(s)
    for _ in range(replays):
        graph.replay()
    torch.cuda.synchronize()


@pytest.mark.parametrize("bf", [0, 1, 2])
def test_dynamic_split_images_equal_the_static_split(gpu, bf):
    # 10 scans of 512 x 512: 10240 linear tiles of 256 points (DAS, identity
    # DMAS) or 20480 of 128 (literal DMAS), over at most 608 CTAs
    cfg = phantom.CONFIGS["dmas2d_512"]
    batch = phantom.make_batch(cfg, 10, first_scan=70)
    grid = cfg.grid()
    tr, ants = dev(batch["traces"]), dev(batch["antennas"])
    P = 512 * 512
    img_d = torch.full((10, P), -1.0, device="cuda")
    pk_d = torch.zeros(10, dtype=torch.int64, device="cuda")
    gpu.uwb_image_batch(bf, tr, ants, grid, cfg.v, cfg.fs, cfg.window, img_d, pk_d)
    torch.cuda.synchronize()
    img_s = torch.full_like(img_d, -1.0)
    pk_s = torch.zeros_like(pk_d)
    _captured(lambda s: gpu.uwb_image_batch(bf, tr, ants, grid, cfg.v, cfg.fs, cfg.window,
                                            img_s, pk_s, stream=s))
    assert torch.equal(img_d, img_s)
    assert torch.equal(pk_d, pk_s)
    # the dynamically split image against the oracle at sampled focal points
    last = img_d[9].cpu().numpy().reshape(512, 512)
    rng = np.random.default_rng(40 + bf)
    pts = rng.integers(0, 512, size=(24, 2))
    ref = np.array([oracle.image(batch["traces"][9], batch["antennas"], grid, cfg.v, cfg.fs,
                                 cfg.window, BF_ORACLE[bf], lo=[x, y, 0], cnt=[1, 1, 1])[0, 0, 0]
                    for x, y in pts])
    got = np.array([last[y, x] for x, y in pts])
    assert np.max(np.abs(got - ref)) <= IMG_TOL * float(last.max())


def test_graph_replayed_localisation_keeps_the_dynamic_split(gpu):
    # 64 scans: the final regions hold about 13k tiles of 128 points, split
    # dynamically over 608 CTAs through the workspace's counters, eagerly and
    # in each of three replays of a captured graph (each replay zeroes them)
    cfg = phantom.CONFIGS["dmas2d_512"]
    batch = phantom.make_batch(cfg, 64, first_scan=80)
    grid = cfg.grid()
    tr, ants = dev(batch["traces"]), dev(batch["antennas"])
    g_rule, _ = rule_pair(gpu)
    B, M, N = batch["traces"].shape
    ws = torch.empty(gpu.uwb_localize_workspace(B, M, N, grid, 2, g_rule), dtype=torch.uint8,
                     device="cuda")
    out_d = torch.empty(B * gpu.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    gpu.uwb_localize_batch(tr, ants, grid, cfg.v, cfg.fs, cfg.window, 2, g_rule, ws, out_d)
    torch.cuda.synchronize()
    res = gpu.results_from_device(out_d)
    assert (res["status"] == 0).all()
    tiles = np.ceil(np.prod(res["roi_hi"] - res["roi_lo"], axis=1) / 128.0).sum()
    assert tiles >= 16 * 608
    out_s = torch.zeros_like(out_d)
    _captured(lambda s: gpu.uwb_localize_batch(tr, ants, grid, cfg.v, cfg.fs, cfg.window, 2,
                                               g_rule, ws, out_s, stream=s), replays=3)
    assert torch.equal(out_d, out_s)


def test_more_launches_in_flight_than_tile_counters(gpu):
    """80 image launches queued on two streams without waiting: the library
    has 64 counters, reuses one only after the launch that used it has
    completed, and splits statically when none is free. Every image must equal
    the one of a lone launch."""
    cfg = phantom.with_changes(phantom.CONFIGS["dmas2d_512"], grid_n=(256, 256, 1))
    batch = phantom.make_batch(cfg, 40, first_scan=150)
    grid = cfg.grid()
    tr, ants = dev(batch["traces"]), dev(batch["antennas"])
    P = 256 * 256
    ref = torch.empty(40, P, device="cuda")
    ref_pk = torch.zeros(40, dtype=torch.int64, device="cuda")
    gpu.uwb_image_batch(0, tr, ants, grid, cfg.v, cfg.fs, cfg.window, ref, ref_pk)
    bufs = [torch.full((40, P), -1.0, device="cuda") for _ in range(16)]
    pks = [torch.zeros(40, dtype=torch.int64, device="cuda") for _ in range(16)]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k in range(80):
        j = k % 16  # buffer j is only ever written on stream j % 2
        gpu.uwb_image_batch(0, tr, ants, grid, cfg.v, cfg.fs, cfg.window, bufs[j], pks[j],
                            stream=streams[k % 2])
    torch.cuda.synchronize()
    for b, p in zip(bufs, pks):
        assert torch.equal(b, ref)
        assert torch.equal(p, ref_pk)
