"""ctypes front end of the FP64 C oracle (``oracle.c``).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package. The CUDA library never does.
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import shutil
import subprocess

import numpy as np

HERE = pathlib.Path(__file__).resolve().parent
LIB_PATH = HERE / "liboracle.so"
SRC = HERE / "oracle.c"

MAX_ITERS = 32
DAS, DMAS = 0, 1
DECIM_MANUAL, DECIM_AUTO = 0, 1
METRIC_HYBRID, METRIC_MEAN, METRIC_VARIANCE, METRIC_HYBRID_UNCLIPPED = 0, 1, 2, 3
STOP_NONE, STOP_METRIC, STOP_MINSIZE, STOP_CAP, STOP_NO_TARGET = 0, 1, 2, 3, 4


def build(force: bool = False) -> pathlib.Path:
    """Compile liboracle.so with gcc (OpenMP if the compiler has it)."""
    if LIB_PATH.exists() and not force and LIB_PATH.stat().st_mtime >= SRC.stat().st_mtime \
            and LIB_PATH.stat().st_mtime >= (HERE / "oracle.h").stat().st_mtime:
        return LIB_PATH
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found for the oracle")
    tmp = LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
    base = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
            str(SRC), "-o", str(tmp), "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("origin", ctypes.c_double * 3), ("pitch", ctypes.c_double * 3)]


class Rule(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("decimation", ctypes.c_int),
                ("min_tumor_diameter", ctypes.c_double), ("metric", ctypes.c_int),
                ("min_segment", ctypes.c_int), ("frame_num", ctypes.c_int),
                ("frame_den", ctypes.c_int), ("max_iters", ctypes.c_int)]


I3 = ctypes.c_int * 3
IT = ctypes.c_int * MAX_ITERS
IT3 = (ctypes.c_int * 3) * MAX_ITERS
DT = ctypes.c_double * MAX_ITERS


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("n_logged", ctypes.c_int), ("stop_reason", ctypes.c_int),
                ("decim", ctypes.c_int), ("offset", I3), ("dcount", I3),
                ("roi_lo", I3), ("roi_hi", I3), ("loc_idx", I3),
                ("loc_xyz", ctypes.c_double * 3), ("peak", ctypes.c_double),
                ("profile_max", ctypes.c_double),
                ("points_evaluated", ctypes.c_longlong),
                ("child", IT), ("n_children", IT), ("box_lo", IT3), ("box_hi", IT3),
                ("metric_top", DT), ("metric_gap", DT), ("between", DT),
                ("within", DT), ("stop_margin", DT)]

    def to_dict(self) -> dict:
        n = self.n_logged
        return {
            "status": self.status, "iters": self.iters, "n_logged": n,
            "stop_reason": self.stop_reason, "decim": self.decim,
            "offset": list(self.offset), "dcount": list(self.dcount),
            "roi_lo": list(self.roi_lo), "roi_hi": list(self.roi_hi),
            "loc_idx": list(self.loc_idx), "loc_xyz": list(self.loc_xyz),
            "peak": self.peak, "profile_max": self.profile_max,
            "points_evaluated": self.points_evaluated,
            "child": list(self.child)[:n], "n_children": list(self.n_children)[:n],
            "box_lo": [list(b) for b in self.box_lo][:n],
            "box_hi": [list(b) for b in self.box_hi][:n],
            "metric_top": list(self.metric_top)[:n],
            "metric_gap": list(self.metric_gap)[:n],
            "between": list(self.between)[:n], "within": list(self.within)[:n],
            "stop_margin": list(self.stop_margin)[:n],
        }


class Path(ctypes.Structure):
    """orc_path: a trajectory for the selection loop to follow (test aid for
    near-ties; see oracle.h)."""
    _fields_ = [("n", ctypes.c_int), ("child", IT), ("cont", IT), ("error", ctypes.c_int),
                ("own_child", IT), ("own_cont", IT), ("taken_metric", DT), ("taken_gap", DT)]


def make_path(child, cont=None) -> Path:
    """child[i] / cont[i] for iteration i + 1; -1 (or None for cont) leaves
    the oracle's own outcome."""
    child = list(child)
    cont = [-1] * len(child) if cont is None else list(cont)
    assert len(child) == len(cont) <= MAX_ITERS
    p = Path()
    p.n = len(child)
    for i, (c, k) in enumerate(zip(child, cont)):
        p.child[i] = int(c)
        p.cont[i] = int(k)
    return p


def _path_log(p: Path, n: int) -> dict:
    return {"error": p.error, "own_child": list(p.own_child)[:n],
            "own_cont": list(p.own_cont)[:n], "taken_metric": list(p.taken_metric)[:n],
            "taken_gap": list(p.taken_gap)[:n]}


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(LIB_PATH))
        fp = ctypes.POINTER(ctypes.c_float)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_image.argtypes = [fp, ctypes.c_int, ctypes.c_int, fp, ctypes.POINTER(Grid),
                                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                ip, ip, ip, dp]
        L.orc_image.restype = ctypes.c_int
        L.orc_image_multistatic.argtypes = [fp, ctypes.c_int, ctypes.c_int, ip, fp, ctypes.c_int,
                                            ctypes.POINTER(Grid), ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, ip,
                                            ip, dp]
        L.orc_image_multistatic.restype = ctypes.c_int
        L.orc_decimation.argtypes = [ctypes.POINTER(Rule), ctypes.POINTER(Grid)]
        L.orc_decimation.restype = ctypes.c_int
        L.orc_lattice_offset.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_lattice_offset.restype = ctypes.c_int
        L.orc_select.argtypes = [dp, ctypes.POINTER(Grid), ctypes.POINTER(Rule),
                                 ctypes.c_int, ctypes.POINTER(Result)]
        L.orc_select.restype = ctypes.c_int
        L.orc_localize.argtypes = [fp, ctypes.c_int, ctypes.c_int, fp, ctypes.POINTER(Grid),
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, ctypes.POINTER(Rule),
                                   ctypes.POINTER(Result)]
        L.orc_localize.restype = ctypes.c_int
        L.orc_hybrid_metric.argtypes = [ctypes.c_double] * 3
        L.orc_hybrid_metric.restype = ctypes.c_double
        L.orc_hybrid_metric_unclipped.argtypes = [ctypes.c_double] * 3
        L.orc_hybrid_metric_unclipped.restype = ctypes.c_double
        L.orc_scatter.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, dp, dp]
        L.orc_scatter.restype = None
        L.orc_localize_multistatic.argtypes = [fp, ctypes.c_int, ctypes.c_int, ip, fp,
                                               ctypes.c_int, ctypes.POINTER(Grid),
                                               ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_int, ctypes.POINTER(Rule),
                                               ctypes.POINTER(Result)]
        L.orc_localize_multistatic.restype = ctypes.c_int
        L.orc_presence.argtypes = [fp, ctypes.c_int, ctypes.c_int, fp, ctypes.POINTER(Grid),
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(Rule), ctypes.c_int, ctypes.POINTER(Result),
                                   ctypes.POINTER(Result)]
        L.orc_presence.restype = ctypes.c_int
        L.orc_localize_progressive.argtypes = L.orc_localize.argtypes
        L.orc_localize_progressive.restype = ctypes.c_int
        L.orc_region_lattice.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip, ip]
        L.orc_region_lattice.restype = None
        pp = ctypes.POINTER(Path)
        L.orc_select_path.argtypes = L.orc_select.argtypes[:4] + [pp, ctypes.POINTER(Result)]
        L.orc_select_path.restype = ctypes.c_int
        L.orc_localize_path.argtypes = L.orc_localize.argtypes[:-1] + [pp,
                                                                       ctypes.POINTER(Result)]
        L.orc_localize_path.restype = ctypes.c_int
        L.orc_localize_progressive_path.argtypes = L.orc_localize_path.argtypes
        L.orc_localize_progressive_path.restype = ctypes.c_int
        L.orc_localize_multistatic_path.argtypes = \
            L.orc_localize_multistatic.argtypes[:-1] + [pp, ctypes.POINTER(Result)]
        L.orc_localize_multistatic_path.restype = ctypes.c_int
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def make_grid(g: dict) -> Grid:
    n = list(g["n"]) + [1] * (3 - len(g["n"]))
    return Grid(int(g["dim"]), I3(*n), (ctypes.c_double * 3)(*g["origin"]),
                (ctypes.c_double * 3)(*g["pitch"]))


def make_rule(mode=DECIM_AUTO, decimation=1, min_tumor_diameter=0.01,
              metric=METRIC_HYBRID, min_segment=4, frame_num=1, frame_den=4,
              max_iters=0) -> Rule:
    return Rule(mode, decimation, min_tumor_diameter, metric, min_segment, frame_num,
                frame_den, max_iters)


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def image(traces, antennas, grid: dict, v, fs, window, beamformer=DAS,
          lo=None, step=None, cnt=None) -> np.ndarray:
    """Energy image over a box lattice; default = the full grid.
    Returns float64 array shaped [cnt_z, cnt_y, cnt_x]."""
    tr, trp = _f32(traces)
    an, anp = _f32(antennas)
    M, N = tr.shape
    n = list(grid["n"]) + [1] * (3 - len(grid["n"]))
    lo = [0, 0, 0] if lo is None else list(lo)
    step = [1, 1, 1] if step is None else list(step)
    cnt = n if cnt is None else list(cnt)
    out = np.zeros(int(np.prod(cnt)), dtype=np.float64)
    g = make_grid(grid)
    st = lib().orc_image(trp, M, N, anp, ctypes.byref(g), float(v), float(fs), int(window),
                         int(beamformer), I3(*lo), I3(*step), I3(*cnt),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != 0:
        raise ValueError(f"orc_image failed: {st}")
    return out.reshape(cnt[2], cnt[1], cnt[0])


def image_multistatic(traces, channels, antennas, grid: dict, v, fs, window, beamformer=DAS,
                      lo=None, step=None, cnt=None) -> np.ndarray:
    """Multistatic energy image; traces [C, N], channels [C, 2] (tx, rx)."""
    tr, trp = _f32(traces)
    an, anp = _f32(antennas)
    ch = np.ascontiguousarray(channels, dtype=np.int32)
    C, N = tr.shape
    M = an.shape[0]
    n = list(grid["n"]) + [1] * (3 - len(grid["n"]))
    lo = [0, 0, 0] if lo is None else list(lo)
    step = [1, 1, 1] if step is None else list(step)
    cnt = n if cnt is None else list(cnt)
    out = np.zeros(int(np.prod(cnt)), dtype=np.float64)
    g = make_grid(grid)
    st = lib().orc_image_multistatic(trp, C, N, ch.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     anp, M, ctypes.byref(g), float(v), float(fs), int(window),
                                     int(beamformer), I3(*lo), I3(*step), I3(*cnt),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != 0:
        raise ValueError(f"orc_image_multistatic failed: {st}")
    return out.reshape(cnt[2], cnt[1], cnt[0])


def decimation(rule: Rule, grid: dict) -> int:
    g = make_grid(grid)
    return lib().orc_decimation(ctypes.byref(rule), ctypes.byref(g))


def lattice_offset(n: int, D: int) -> int:
    return lib().orc_lattice_offset(n, D)


def select(profile_norm: np.ndarray, grid: dict, rule: Rule, D: int,
           path: Path | None = None) -> dict:
    """Selection loop on a normalised decimated profile. With a path, the
    loop follows it and the result carries the path log under "path"."""
    e = np.ascontiguousarray(profile_norm, dtype=np.float64).ravel()
    g = make_grid(grid)
    res = Result()
    st = lib().orc_select_path(e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               ctypes.byref(g), ctypes.byref(rule), int(D),
                               None if path is None else ctypes.byref(path), ctypes.byref(res))
    if st != 0 and (path is None or path.error == 0):
        raise ValueError(f"orc_select failed: {st}")
    out = res.to_dict()
    if path is not None:
        out["path"] = _path_log(path, res.n_logged)
    return out


def _with_path(res: Result, path: Path | None) -> dict:
    out = res.to_dict()
    if path is not None:
        out["path"] = _path_log(path, res.n_logged)
    return out


def localize(traces, antennas, grid: dict, v, fs, window, beamformer=DAS,
             rule: Rule | None = None, path: Path | None = None) -> dict:
    """The framework (orc_localize); with a path, along that trajectory
    (orc_localize_path), the path log under "path"."""
    tr, trp = _f32(traces)
    an, anp = _f32(antennas)
    M, N = tr.shape
    rule = make_rule() if rule is None else rule
    g = make_grid(grid)
    res = Result()
    lib().orc_localize_path(trp, M, N, anp, ctypes.byref(g), float(v), float(fs), int(window),
                            int(beamformer), ctypes.byref(rule),
                            None if path is None else ctypes.byref(path), ctypes.byref(res))
    return _with_path(res, path)


def localize_progressive(traces, antennas, grid: dict, v, fs, window, beamformer=DAS,
                         rule: Rule | None = None, path: Path | None = None) -> dict:
    """The framework with progressive re-evaluation (orc_localize_progressive);
    with a path, along that trajectory."""
    tr, trp = _f32(traces)
    an, anp = _f32(antennas)
    M, N = tr.shape
    g = make_grid(grid)
    res = Result()
    rule = make_rule() if rule is None else rule
    st = lib().orc_localize_progressive_path(trp, M, N, anp, ctypes.byref(g), float(v),
                                             float(fs), int(window), int(beamformer),
                                             ctypes.byref(rule),
                                             None if path is None else ctypes.byref(path),
                                             ctypes.byref(res))
    out = _with_path(res, path)
    out["status"] = st if st != 0 else out["status"]
    return out


def region_lattice(lo: int, hi: int, c0: int):
    """(first index, step, count) of orc_region_lattice."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib().orc_region_lattice(int(lo), int(hi), int(c0), ctypes.byref(a), ctypes.byref(b),
                             ctypes.byref(c))
    return a.value, b.value, c.value


def presence(traces, antennas, grid: dict, v, fs, window, beamformer=DAS, rule: Rule | None = None,
             decimation2: int = 1):
    """Two-decimation tumour-presence test: (present, result1, result2)."""
    tr, trp = _f32(traces)
    an, anp = _f32(antennas)
    M, N = tr.shape
    rule = make_rule() if rule is None else rule
    g = make_grid(grid)
    r1, r2 = Result(), Result()
    st = lib().orc_presence(trp, M, N, anp, ctypes.byref(g), float(v), float(fs), int(window),
                            int(beamformer), ctypes.byref(rule), int(decimation2), ctypes.byref(r1),
                            ctypes.byref(r2))
    if st < 0:
        raise ValueError(f"orc_presence failed: {st}")
    return bool(st), r1.to_dict(), r2.to_dict()


def localize_multistatic(traces, channels, antennas, grid: dict, v, fs, window, beamformer=DAS,
                         rule: Rule | None = None, path: Path | None = None) -> dict:
    tr, trp = _f32(traces)
    an, anp = _f32(antennas)
    ch = np.ascontiguousarray(channels, dtype=np.int32)
    C, N = tr.shape
    rule = make_rule() if rule is None else rule
    g = make_grid(grid)
    res = Result()
    lib().orc_localize_multistatic_path(trp, C, N,
                                        ch.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), anp,
                                        an.shape[0], ctypes.byref(g), float(v), float(fs),
                                        int(window), int(beamformer), ctypes.byref(rule),
                                        None if path is None else ctypes.byref(path),
                                        ctypes.byref(res))
    return _with_path(res, path)


def hybrid_metric(mean_i: float, var_i: float, var_prev: float) -> float:
    return lib().orc_hybrid_metric(mean_i, var_i, var_prev)


def hybrid_metric_unclipped(mean_i: float, var_i: float, var_prev: float) -> float:
    return lib().orc_hybrid_metric_unclipped(mean_i, var_i, var_prev)


def scatter(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    w = ctypes.c_double()
    bb = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    lib().orc_scatter(a.ctypes.data_as(dp), len(a), b.ctypes.data_as(dp), len(b),
                      ctypes.byref(w), ctypes.byref(bb))
    return w.value, bb.value


def num_threads() -> int:
    return lib().orc_num_threads()
