"""Helpers shared by the GPU parity tests: device marshalling and the
comparison rules between the CUDA path and the FP64 oracle.

Tolerances:
* images: |gpu - oracle| <= 1e-4 * max(oracle), element by element (float32
  arithmetic against float64);
* decisions (chosen child, framed boxes, stop test, final argmax) are integers
  and must be equal, except where the oracle's own decision margin is below
  the image tolerance: there two answers are both correct, and the GPU's is
  checked for validity instead (its metric or energy within tolerance of the
  oracle's best), and nothing after it is compared.
"""
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


def compare_localize(g: dict, o: dict, energy_at=None) -> dict:
    """Checks one scan's GPU result against the oracle's. energy_at(idx) gives
    the oracle energy at a focal point (for validating an argmax near-tie).
    Returns a summary with the smallest decision margin seen."""
    assert g["status"] == o["status"], (g["status"], o["status"])
    for key in ("decim", "offset", "dcount"):
        assert g[key] == o[key], key
    if o["status"] != 0:
        return {"tie": False, "min_margin": None}
    if o["stop_reason"] == oracle.STOP_NO_TARGET:
        assert g["stop_reason"] == o["stop_reason"] and g["loc_idx"] == [-1, -1, -1]
        return {"tie": False, "min_margin": None}
    min_margin = float("inf")
    for i in range(o["n_logged"]):
        gap = o["metric_gap"][i]
        min_margin = min(min_margin, gap)
        if gap < MARGIN:
            # near-tie: the GPU's child must score within tolerance of the best
            assert i < g["n_logged"]
            assert g["metric_top"][i] >= o["metric_top"][i] * (1 - 1e-3) - 1e-12
            return {"tie": True, "min_margin": min_margin, "at": ("metric", i)}
        assert g["child"][i] == o["child"][i], ("child", i, g["child"], o["child"])
        assert g["box_lo"][i] == o["box_lo"][i] and g["box_hi"][i] == o["box_hi"][i], ("box", i)
        np.testing.assert_allclose(g["metric_top"][i], o["metric_top"][i], rtol=2e-3, atol=1e-9)
        sm = o["stop_margin"][i]
        min_margin = min(min_margin, sm)
        if sm < MARGIN:
            return {"tie": True, "min_margin": min_margin, "at": ("stop", i)}
    assert g["n_logged"] == o["n_logged"]
    assert g["iters"] == o["iters"] and g["stop_reason"] == o["stop_reason"]
    assert g["roi_lo"] == o["roi_lo"] and g["roi_hi"] == o["roi_hi"]
    assert g["points_evaluated"] == o["points_evaluated"]
    np.testing.assert_allclose(g["profile_max"], o["profile_max"], rtol=IMG_TOL)
    tie = False
    if g["loc_idx"] != o["loc_idx"]:
        # both argmaxes are right only if the energies agree within tolerance
        assert energy_at is not None, ("location", g["loc_idx"], o["loc_idx"])
        e_g = energy_at(g["loc_idx"])
        assert abs(e_g - o["peak"]) <= IMG_TOL * o["peak"], ("location", g["loc_idx"],
                                                             o["loc_idx"], e_g, o["peak"])
        tie = True
    np.testing.assert_allclose(g["peak"], o["peak"], rtol=IMG_TOL)
    if not tie:
        np.testing.assert_allclose(g["loc_xyz"], o["loc_xyz"], rtol=1e-12, atol=1e-15)
    return {"tie": tie, "min_margin": min_margin}
