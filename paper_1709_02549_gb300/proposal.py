"""Training and evaluation of the learned segment proposal on scans the
method itself generates (not part of the paper).

Data: seeded 2-D scans of a workload (default: 32-antenna ring, 512 x 512
grid over 12 cm, 2048 samples, 50 clutter scatterers, 15 dB SNR). Each scan
is localised by the plain framework (Eq. 5 selection, identity-form DMAS), and
its located point labels two coarse DAS maps: the whole grid (label = the 4 x 4
segment holding the point) and that segment (label = the sub-segment holding
it). The network is trained on both levels with the library's own forward,
backward and Adam kernels.

    python -m paper_1709_02549_gb300.proposal train --scans 100000 --out W.npz
    python -m paper_1709_02549_gb300.proposal evaluate --weights W.npz --scans 4096

Weights are stored as an .npz of the float32 parameter vector (``theta``) with
the training record (workload, seeds, threshold, accuracies) as JSON text.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import pathlib
import sys
import time

import numpy as np

ROOT = pathlib.Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

import phantom  # noqa: E402  (seeded input generator)

SEG = 4
MAP = 32
DEFAULT_WEIGHTS = pathlib.Path(__file__).resolve().parent / "weights" / "proposal_dmas2d_512.npz"
TRAIN_FIRST_SCAN = 1_000_000      # training scans never overlap the benchmark's seeds
VALID_FIRST_SCAN = 2_000_000
EVAL_FIRST_SCAN = 3_000_000


def _gen(args):
    name, n, first = args
    b = phantom.make_batch(phantom.CONFIGS[name], n, first)
    return b["traces"], b["tumors"]


def scan_chunks(name: str, n_scans: int, first_scan: int, chunk: int = 1024, workers: int = 0):
    """Yields (traces [c, M, N] float32, tumours) chunks of seeded scans,
    generated in a spawned process pool (safe next to a CUDA context)."""
    import os
    workers = workers or min(16, os.cpu_count() or 1)
    sub = max(1, chunk // workers)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for c0 in range(0, n_scans, chunk):
            c = min(chunk, n_scans - c0)
            jobs = [(name, min(sub, c - k), first_scan + c0 + k) for k in range(0, c, sub)]
            parts = pool.map(_gen, jobs)
            yield (np.concatenate([p[0] for p in parts]),
                   [t for p in parts for t in p[1]])


def segment_labels(loc_xy: np.ndarray, n: int):
    """Level-1 segment, level-2 region origin and level-2 sub-segment of each
    located point (x, y) on an n x n grid."""
    side1 = n // SEG
    sx, sy = loc_xy[:, 0] // side1, loc_xy[:, 1] // side1
    s1 = (SEG * sy + sx).astype(np.int32)
    lo = np.stack([sx * side1, sy * side1], 1).astype(np.int32)
    side2 = side1 // SEG
    tx, ty = (loc_xy[:, 0] - lo[:, 0]) // side2, (loc_xy[:, 1] - lo[:, 1]) // side2
    s2 = (SEG * ty + tx).astype(np.int32)
    return s1, lo, s2


class Workload:
    """Device-side helpers for one workload: framework labels and coarse maps."""

    def __init__(self, name: str = "dmas2d_512"):
        import torch
        import paper_1709_02549_gb300 as u
        self.u, self.torch = u, torch
        self.cfg = phantom.CONFIGS[name]
        self.name = name
        self.grid = self.cfg.grid()
        self.n = self.grid["n"][0]
        self.ants = torch.from_numpy(phantom.antenna_positions(self.cfg).astype(np.float32)).cuda()
        self.rule = u.uwb_default_rule()

    def framework(self, traces, beamformer=None):
        """Plain framework localisation (Eq. 5): result records on the host."""
        u, torch = self.u, self.torch
        bf = u.UWB_DMAS if beamformer is None else beamformer
        B, M, N = traces.shape
        ws = torch.empty(u.uwb_localize_workspace(B, M, N, self.grid, bf, self.rule),
                         dtype=torch.uint8, device="cuda")
        out = torch.empty(B * u.RESULT_BYTES, dtype=torch.uint8, device="cuda")
        u.uwb_localize_batch(traces, self.ants, self.grid, self.cfg.v, self.cfg.fs,
                             self.cfg.window, bf, self.rule, ws, out)
        return u.results_from_device(out)

    def maps(self, traces, side, region_lo=None):
        u, torch = self.u, self.torch
        B = traces.shape[0]
        m = torch.empty(B, MAP, MAP, device="cuda")
        ws = None
        if region_lo is not None:
            ws = torch.empty(max(256, u.uwb_coarse_maps_workspace(B)), dtype=torch.uint8,
                             device="cuda")
        u.uwb_coarse_maps(traces, self.ants, self.grid, self.cfg.v, self.cfg.fs, self.cfg.window,
                          side, m, region_lo, ws)
        return m

    def learned(self, traces, packed, threshold, beamformer=None, levels=2):
        u, torch = self.u, self.torch
        bf = u.UWB_DMAS_LITERAL if beamformer is None else beamformer
        B = traces.shape[0]
        ws = torch.empty(u.uwb_localize_learned_workspace(B, self.grid, self.rule),
                         dtype=torch.uint8, device="cuda")
        out = torch.empty(B * u.RESULT_BYTES, dtype=torch.uint8, device="cuda")
        u.uwb_localize_learned(traces, self.ants, self.grid, self.cfg.v, self.cfg.fs,
                               self.cfg.window, bf, self.rule, packed, threshold, levels, ws, out)
        return u.results_from_device(out)


def build_dataset(wl: Workload, n_scans: int, first_scan: int, chunk: int = 1024, log=print):
    """Coarse maps of both levels with their framework labels (device tensors)."""
    torch = wl.torch
    maps, labels = [], []
    t0 = time.time()
    for traces, _ in scan_chunks(wl.name, n_scans, first_scan, chunk):
        tr = torch.from_numpy(traces).cuda()
        rec = wl.framework(tr)
        loc = np.stack([rec["loc_idx"][:, 0], rec["loc_idx"][:, 1]], 1).astype(np.int64)
        ok = (rec["status"] == 0) & (loc[:, 0] >= 0)
        s1, lo, s2 = segment_labels(np.maximum(loc, 0), wl.n)
        m1 = wl.maps(tr, wl.n)
        m2 = wl.maps(tr, wl.n // SEG, torch.from_numpy(lo).cuda())
        keep = torch.from_numpy(ok).cuda()
        maps += [m1[keep], m2[keep]]
        labels += [torch.from_numpy(s1).cuda()[keep], torch.from_numpy(s2).cuda()[keep]]
        done = sum(x.shape[0] for x in maps) // 2
        log(f"  {done} scans labelled ({time.time() - t0:.0f} s)")
    return torch.cat(maps), torch.cat(labels).int()


N_PARAMS = 18849
SIZES = [(32, 9), (32,), (32, 9, 32), (32,), (32, 9, 32), (32,), (32,), (1,)]


def init_theta(seed: int) -> np.ndarray:
    """He-normal convolution weights, zero biases, a small head; the layout of
    the C ABI's parameter vector (W1, b1, W2, b2, W3, b3, wh, bh)."""
    rng = np.random.Generator(np.random.Philox(seed))
    scales = [np.sqrt(2.0 / 9), 0.0, np.sqrt(2.0 / 288), 0.0, np.sqrt(2.0 / 288), 0.0,
              np.sqrt(1.0 / 32), 0.0]
    parts = [rng.normal(0.0, sc, sh) if sc > 0 else np.zeros(sh) for sc, sh in zip(scales, SIZES)]
    theta = np.concatenate([x.ravel() for x in parts]).astype(np.float32)
    assert theta.size == N_PARAMS
    return theta


def _dihedral(torch, maps, labels, k: int):
    """The k-th of the 8 symmetries of the square applied to [B, 32, 32] maps
    and to their 4 x 4 segment labels."""
    grid = torch.arange(16, device=maps.device).reshape(4, 4)
    if k >= 4:
        maps, grid = maps.flip(-1), grid.flip(-1)
    r = k % 4
    maps = torch.rot90(maps, r, (-2, -1))
    grid = torch.rot90(grid, r, (-2, -1))
    # new position q holds old segment grid[q]: old label s moves to the q with grid[q] == s
    where = torch.empty(16, dtype=torch.long, device=maps.device)
    where[grid.reshape(-1)] = torch.arange(16, device=maps.device)
    return maps.contiguous(), where[labels.long()].int()


def train(wl: Workload, maps, labels, epochs: int = 6, batch: int = 256, lr: float = 2e-3,
          seed: int = 1709, log=print):
    """Adam on shuffled minibatches (each under a random symmetry of the square)
    with a cosine learning-rate decay to 2 % of `lr`; returns (theta, packed)
    device tensors."""
    import math
    u, torch = wl.u, wl.torch
    theta = torch.from_numpy(init_theta(seed)).cuda()
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    packed = torch.zeros(u.CNN_PACKED_BYTES, dtype=torch.uint8, device="cuda")
    u.uwb_cnn_pack(theta, packed)
    ws = torch.empty(u.uwb_cnn_train_workspace(batch), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(1, device="cuda")
    n = maps.shape[0]
    per_epoch = n // batch
    total = epochs * per_epoch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    rng = np.random.Generator(np.random.Philox(seed))
    step, run, t0 = 0, 0.0, time.time()
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        for k in range(per_epoch):
            idx = perm[k * batch:(k + 1) * batch]
            mb, lb = _dihedral(torch, maps[idx], labels[idx], int(rng.integers(8)))
            step += 1
            lr_t = lr * (0.02 + 0.49 * (1.0 + math.cos(math.pi * step / total)))
            u.uwb_cnn_train_step(theta, m, v, packed, mb, lb, step, lr_t, loss, ws)
            if step % 200 == 0 or step == total:
                run = loss.item()
                log(f"  epoch {ep + 1}/{epochs} step {step}/{total} loss {run:.4f} "
                    f"({time.time() - t0:.0f} s)")
    torch.cuda.synchronize()
    return theta, packed


def map_accuracy(wl: Workload, packed, maps, labels):
    """Per-map top-1 accuracy and confidence (largest softmax probability)."""
    u, torch = wl.u, wl.torch
    scores = torch.empty(maps.shape[0], 16, device="cuda")
    u.uwb_cnn_forward(packed, maps.contiguous(), scores)
    p = torch.softmax(scores.double(), 1)
    conf, top = p.max(1)
    return (top.int() == labels).cpu().numpy(), conf.cpu().numpy()


def compare(wl: Workload, packed, threshold: float, chunks, beamformer=None, framework=None):
    """Learned localisation against the plain framework (same final beamformer)
    on chunks of scans [(traces, tumours), ...]: agreement, fallback rate,
    points evaluated, localisation errors against the drawn tumour."""
    u, torch = wl.u, wl.torch
    bf = u.UWB_DMAS_LITERAL if beamformer is None else beamformer
    agree, fallback, pts_l, pts_f, err_l, err_f = [], [], [], [], [], []
    g = wl.grid
    n_scans = 0
    for ci, (traces, tumors) in enumerate(chunks):
        n_scans += traces.shape[0]
        tr = torch.from_numpy(traces).cuda()
        rl = wl.learned(tr, packed, threshold, bf)
        rf = framework[ci] if framework is not None else wl.framework(tr, bf)
        agree.append(np.all(rl["loc_idx"][:, :2] == rf["loc_idx"][:, :2], axis=1))
        fallback.append(rl["stop_reason"] != u.UWB_STOP_LEARNED)
        pts_l.append(rl["points_evaluated"])
        pts_f.append(rf["points_evaluated"])
        truth = np.array([t[0][:2] for t in tumors])
        for rec, out in ((rl, err_l), (rf, err_f)):
            xy = np.stack([g["origin"][a] + rec["loc_idx"][:, a] * g["pitch"][a]
                           for a in range(2)], 1)
            out.append(np.linalg.norm(xy - truth, axis=1) * 1e3)
    cat = np.concatenate
    return {"scans": int(n_scans), "threshold": float(threshold),
            "agreement": float(cat(agree).mean()), "fallback": float(cat(fallback).mean()),
            "points_learned": float(cat(pts_l).mean()), "points_framework": float(cat(pts_f).mean()),
            "err_mm_learned": float(cat(err_l).mean()), "err_mm_framework": float(cat(err_f).mean()),
            "err_mm_learned_p99": float(np.percentile(cat(err_l), 99)),
            "err_mm_framework_p99": float(np.percentile(cat(err_f), 99))}


THRESHOLDS = [0.5, 0.6, 0.7, 0.8, 0.9, 0.95, 0.98, 0.99, 0.995]


def pick_threshold(wl: Workload, packed, chunks, max_disagree: float, log=print):
    """Smallest candidate confidence threshold whose learned locations differ
    from the framework's on at most `max_disagree` of the validation scans."""
    torch = wl.torch
    framework = [wl.framework(torch.from_numpy(tr).cuda(), wl.u.UWB_DMAS_LITERAL)
                 for tr, _ in chunks]
    rows = []
    for th in THRESHOLDS:
        r = compare(wl, packed, th, chunks, framework=framework)
        rows.append(r)
        log(f"  threshold {th}: agreement {r['agreement']:.4f} fallback {r['fallback']:.4f} "
            f"points {r['points_learned']:.0f} vs {r['points_framework']:.0f}")
        if 1.0 - r["agreement"] <= max_disagree:
            return th, rows
    return THRESHOLDS[-1], rows


def save(path, theta, record: dict):
    path = pathlib.Path(path)
    path.parent.mkdir(parents=True, exist_ok=True)
    np.savez(path, theta=np.asarray(theta, np.float32), record=np.array(json.dumps(record)))


def load(path=DEFAULT_WEIGHTS):
    """(theta float32 [18849], training record dict)."""
    with np.load(path) as z:
        return z["theta"].astype(np.float32), json.loads(str(z["record"]))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--workload", default="dmas2d_512")
    t.add_argument("--scans", type=int, default=100_000)
    t.add_argument("--valid", type=int, default=2048)
    t.add_argument("--epochs", type=int, default=6)
    t.add_argument("--batch", type=int, default=256)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--seed", type=int, default=1709)
    t.add_argument("--max-disagree", type=float, default=0.002)
    t.add_argument("--out", default=str(DEFAULT_WEIGHTS))
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", default=str(DEFAULT_WEIGHTS))
    e.add_argument("--scans", type=int, default=4096)
    e.add_argument("--threshold", type=float, default=None)
    args = ap.parse_args(argv)

    import torch
    import paper_1709_02549_gb300 as u
    wl = Workload(args.workload if args.cmd == "train" else "dmas2d_512")
    if args.cmd == "train":
        t0 = time.time()
        print(f"labelling {args.scans} training scans", flush=True)
        maps, labels = build_dataset(wl, args.scans, TRAIN_FIRST_SCAN,
                                     log=lambda s: print(s, flush=True))
        t_data = time.time() - t0
        print(f"training on {maps.shape[0]} maps", flush=True)
        t1 = time.time()
        theta, packed = train(wl, maps, labels, args.epochs, args.batch, args.lr, args.seed,
                              log=lambda s: print(s, flush=True))
        t_train = time.time() - t1
        vmaps, vlabels = build_dataset(wl, args.valid, VALID_FIRST_SCAN, log=lambda s: None)
        acc, conf = map_accuracy(wl, packed, vmaps, vlabels)
        vchunks = list(scan_chunks(wl.name, args.valid, VALID_FIRST_SCAN))
        th, rows = pick_threshold(wl, packed, vchunks, args.max_disagree,
                                  log=lambda s: print(s, flush=True))
        record = {"workload": args.workload, "train_scans": args.scans,
                  "train_first_scan": TRAIN_FIRST_SCAN, "valid_scans": args.valid,
                  "valid_first_scan": VALID_FIRST_SCAN, "epochs": args.epochs,
                  "batch": args.batch, "lr": args.lr, "seed": args.seed,
                  "threshold": th, "valid_map_accuracy": float(acc.mean()),
                  "valid_threshold_sweep": rows, "seconds_data": round(t_data, 1),
                  "seconds_train": round(t_train, 1), "max_disagree": args.max_disagree}
        save(args.out, theta.cpu().numpy(), record)
        print(json.dumps({k: v for k, v in record.items() if k != "valid_threshold_sweep"}),
              flush=True)
    else:
        theta, record = load(args.weights)
        th = record["threshold"] if args.threshold is None else args.threshold
        tt = torch.from_numpy(theta).cuda()
        packed = torch.zeros(u.CNN_PACKED_BYTES, dtype=torch.uint8, device="cuda")
        u.uwb_cnn_pack(tt, packed)
        r = compare(wl, packed, th, scan_chunks(wl.name, args.scans, EVAL_FIRST_SCAN))
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
