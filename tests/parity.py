"""Helpers shared by the GPU parity tests: device marshalling and the
comparison rules between the CUDA path and the FP64 oracle.

Tolerances:
* images: |gpu - oracle| <= 1e-4 * max(oracle), element by element (float32
  arithmetic against float64);
* decisions (chosen child, framed boxes, stop test, final region, argmax) are
  integers and must be equal. Where the oracle's own decision margin is below
  the image tolerance (two children whose Eq. 5 metrics differ by less than
  1e-4 relative, or an Eq. 6-7 test whose B or W differs from the previous
  iteration's by less than 1e-4 relative), both outcomes are correct and the
  GPU may take the other one. The oracle is then replayed along the GPU's
  whole trajectory (orc_path): every step where the GPU departed from the
  oracle's own choice must be such a near-tie by the oracle's FP64 margins,
  and everything else (framed boxes, stop decisions, final region, point
  count, location) must equal the replay's. A location that differs is
  accepted only where the oracle's energies at the two points agree within
  the image tolerance.
Every comparison is tallied per test (scans compared, near-ties taken at a
child, a stop test or the argmax); conftest prints the tallies.
"""
import collections

import numpy as np
import torch

import oracle

IMG_TOL = 1e-4
MARGIN = 1e-4

BF_ORACLE = {0: oracle.DAS, 1: oracle.DMAS, 2: oracle.DMAS}


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def gpu_image_batch(uwb, bf, traces, ants, grid, v, fs, W, with_peak=True):
    traces = np.asarray(traces, np.float32)
    if traces.ndim == 2:
        traces = traces[None]
    B = traces.shape[0]
    n = list(grid["n"]) + [1] * (3 - len(grid["n"]))
    P = int(np.prod(n))
    img = torch.full((B, P), -1.0, device="cuda")
    peak = torch.zeros(B, dtype=torch.int64, device="cuda") if with_peak else None
    uwb.uwb_image_batch(bf, dev(traces), dev(ants), grid, v, fs, W, img, peak)
    torch.cuda.synchronize()
    out = img.cpu().numpy().reshape(B, n[2], n[1], n[0])
    return out, (peak.cpu().numpy() if with_peak else None)


def gpu_localize_batch(uwb, bf, traces, ants, grid, v, fs, W, rule, image=False):
    traces = np.asarray(traces, np.float32)
    if traces.ndim == 2:
        traces = traces[None]
    B, M, N = traces.shape
    ws_bytes = uwb.uwb_localize_workspace(B, M, N, grid, bf, rule)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = torch.empty(B * uwb.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    n = list(grid["n"]) + [1] * (3 - len(grid["n"]))
    img = torch.full((B, int(np.prod(n))), -1.0, device="cuda") if image else None
    uwb.uwb_localize_batch(dev(traces), dev(ants), grid, v, fs, W, bf, rule, ws, out, img)
    torch.cuda.synchronize()
    recs = uwb.results_from_device(out)
    res = [record_to_dict(r) for r in recs]
    if image:
        return res, img.cpu().numpy().reshape(B, n[2], n[1], n[0])
    return res


def record_to_dict(r) -> dict:
    n = int(r["n_logged"])
    return {
        "status": int(r["status"]), "iters": int(r["iters"]), "n_logged": n,
        "stop_reason": int(r["stop_reason"]), "decim": int(r["decim"]),
        "offset": [int(x) for x in r["offset"]], "dcount": [int(x) for x in r["dcount"]],
        "roi_lo": [int(x) for x in r["roi_lo"]], "roi_hi": [int(x) for x in r["roi_hi"]],
        "loc_idx": [int(x) for x in r["loc_idx"]], "loc_xyz": [float(x) for x in r["loc_xyz"]],
        "peak": float(r["peak"]), "profile_max": float(r["profile_max"]),
        "points_evaluated": int(r["points_evaluated"]),
        "child": [int(x) for x in r["child"][:n]],
        "n_children": [int(x) for x in r["n_children"][:n]],
        "box_lo": [[int(y) for y in x] for x in r["box_lo"][:n]],
        "box_hi": [[int(y) for y in x] for x in r["box_hi"][:n]],
        "metric_top": [float(x) for x in r["metric_top"][:n]],
        "metric_gap": [float(x) for x in r["metric_gap"][:n]],
        "between": [float(x) for x in r["between"][:n]],
        "within": [float(x) for x in r["within"][:n]],
        "stop_margin": [float(x) for x in r["stop_margin"][:n]],
    }


def rule_pair(uwb, **kw):
    """The same decision rule for the GPU library and the oracle."""
    g = uwb.uwb_default_rule(**kw)
    o = oracle.make_rule(mode=g.mode, decimation=g.decimation,
                         min_tumor_diameter=g.min_tumor_diameter, metric=g.metric,
                         min_segment=g.min_segment, frame_num=g.frame_num,
                         frame_den=g.frame_den, max_iters=g.max_iters)
    return g, o


def assert_image_close(gpu, ref, tol=IMG_TOL, what="image"):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    err = float(np.max(np.abs(gpu - ref))) if ref.size else 0.0
    assert err <= tol * max(scale, 1e-300), f"{what}: max error {err:.3e} vs {tol} * {scale:.3e}"
    return err / max(scale, 1e-300)


class OracleScan:
    """One scan as the oracle sees it: its localisation along the oracle's own
    trajectory or along a given one, and the energy at single focal points.
    bf is the library's beamformer code (0 DAS, 1 DMAS, 2 literal DMAS);
    channels selects the multistatic oracle, progressive the progressive
    variant."""

    def __init__(self, traces, antennas, grid, v, fs, window, bf, rule, channels=None,
                 progressive=False):
        self.traces = np.asarray(traces, np.float32)
        self.antennas = np.asarray(antennas, np.float32)
        self.grid, self.v, self.fs, self.window = grid, v, fs, window
        self.obf = BF_ORACLE[bf]
        self.rule = rule
        self.channels = channels
        self.progressive = progressive

    def localize(self, path=None) -> dict:
        args = (self.grid, self.v, self.fs, self.window, self.obf, self.rule)
        if self.channels is not None:
            return oracle.localize_multistatic(self.traces, self.channels, self.antennas, *args,
                                               path=path)
        if self.progressive:
            return oracle.localize_progressive(self.traces, self.antennas, *args, path=path)
        return oracle.localize(self.traces, self.antennas, *args, path=path)

    def energy_at(self, idx) -> float:
        if self.channels is not None:
            img = oracle.image_multistatic(self.traces, self.channels, self.antennas, self.grid,
                                           self.v, self.fs, self.window, self.obf, lo=idx,
                                           cnt=[1, 1, 1])
        else:
            img = oracle.image(self.traces, self.antennas, self.grid, self.v, self.fs,
                               self.window, self.obf, lo=idx, cnt=[1, 1, 1])
        return float(img[0, 0, 0])


# tallies per test node id: scans, child / stop / argmax near-ties, replays
TIE_LOG: dict = collections.defaultdict(collections.Counter)
CURRENT_TEST = "?"


def _trajectory(r: dict):
    return (r["child"], r["n_logged"], r["iters"], r["stop_reason"])


def path_of(g: dict) -> oracle.Path:
    """The GPU's trajectory as an orc_path: its children, and the continue /
    stop outcome of every Eq. 6-7 test it made (from the second iteration)."""
    n = g["n_logged"]
    cont = [-1] + [1] * max(0, n - 1)
    if n >= 2 and g["stop_reason"] == oracle.STOP_METRIC:
        cont[n - 1] = 0
    return oracle.make_path(g["child"], cont[:n])


def compare_localize(g: dict, scan: OracleScan, o: dict | None = None) -> dict:
    """Checks one scan's GPU record against the oracle (o: the oracle's own
    result, computed if not given). Returns the near-ties it resolved."""
    o = scan.localize() if o is None else o
    tally = TIE_LOG[CURRENT_TEST]
    tally["scans"] += 1
    out = {"tie": False, "child": 0, "stop": 0, "argmax": 0, "replayed": False}
    assert g["status"] == o["status"], (g["status"], o["status"])
    for key in ("decim", "offset", "dcount"):
        assert g[key] == o[key], key
    if o["status"] != 0:
        return out
    np.testing.assert_allclose(g["profile_max"], o["profile_max"], rtol=IMG_TOL)
    if o["stop_reason"] == oracle.STOP_NO_TARGET:
        assert g["stop_reason"] == o["stop_reason"] and g["loc_idx"] == [-1, -1, -1]
        return out
    if _trajectory(g) != _trajectory(o):
        # the GPU took another path: replay the oracle along it, and accept
        # each departure only at a near-tie of the oracle's own margins
        path = path_of(g)
        r = scan.localize(path)
        log = r["path"]
        assert log["error"] == 0, ("GPU chose a child that is not a candidate",
                                   log["error"], g["child"])
        for i in range(min(g["n_logged"], r["n_logged"])):
            if log["own_child"][i] != g["child"][i]:
                assert log["taken_gap"][i] < MARGIN, ("child", i, g["child"], o["child"],
                                                      log["taken_gap"][i])
                out["child"] += 1
            if i >= 1 and log["own_cont"][i] != path.cont[i]:
                assert abs(r["stop_margin"][i]) < MARGIN, ("stop", i, r["stop_margin"][i])
                out["stop"] += 1
        assert out["child"] + out["stop"] > 0, "replay along the GPU path changed nothing"
        out["replayed"] = True
        o = r
    assert g["n_logged"] == o["n_logged"], (g["n_logged"], o["n_logged"])
    assert g["iters"] == o["iters"] and g["stop_reason"] == o["stop_reason"]
    for i in range(o["n_logged"]):
        assert g["child"][i] == o["child"][i], ("child", i, g["child"], o["child"])
        assert g["n_children"][i] == o["n_children"][i], ("candidates", i)
        assert g["box_lo"][i] == o["box_lo"][i] and g["box_hi"][i] == o["box_hi"][i], ("box", i)
        np.testing.assert_allclose(g["metric_top"][i], o["metric_top"][i], rtol=2e-3, atol=1e-9)
    assert g["roi_lo"] == o["roi_lo"] and g["roi_hi"] == o["roi_hi"]
    assert g["points_evaluated"] == o["points_evaluated"]
    if g["loc_idx"] != o["loc_idx"]:
        # both argmaxes are right only if the energies agree within tolerance
        e_g = scan.energy_at(g["loc_idx"])
        assert abs(e_g - o["peak"]) <= IMG_TOL * o["peak"], ("location", g["loc_idx"],
                                                             o["loc_idx"], e_g, o["peak"])
        out["argmax"] += 1
    else:
        np.testing.assert_allclose(g["loc_xyz"], o["loc_xyz"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(g["peak"], o["peak"], rtol=IMG_TOL)
    out["tie"] = bool(out["child"] or out["stop"] or out["argmax"])
    for key in ("child", "stop", "argmax"):
        tally[key] += out[key]
    tally["replayed"] += out["replayed"]
    return out
