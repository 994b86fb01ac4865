"""Python binding of libuwb.so (segment-search confocal UWB imaging on GB300).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. Functions carry the C names of ``include/uwb.h`` and take torch CUDA
tensors (float32, contiguous) for the arrays; ``grid`` is a dict
``{"dim", "n", "origin", "pitch"}`` and ``rule`` a :class:`UwbRule`.
There is no CPU fallback: if the library is not built, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import pathlib

import numpy as np

__all__ = [
    "UWB_OK", "UWB_DAS", "UWB_DMAS", "UWB_DMAS_LITERAL", "UwbGrid", "UwbRule", "UwbResult",
    "RESULT_DTYPE", "lib", "make_grid", "uwb_default_rule", "uwb_decimation", "uwb_das_image",
    "uwb_dmas_image", "uwb_image_batch", "uwb_localize_workspace", "uwb_localize",
    "uwb_localize_batch", "uwb_device_status", "uwb_last_error", "results_from_device",
    "uwb_phase_timing", "uwb_phase_times", "uwb_localize_batch_noalloc",
    "uwb_localize_host_workspace", "uwb_localize_host", "uwb_presence_workspace",
    "uwb_presence_batch", "uwb_image_multistatic_batch", "uwb_localize_multistatic_workspace",
    "uwb_localize_multistatic_batch", "UwbScan", "UwbPlan", "UWB_F32", "UWB_F16", "UWB_BF16",
    "uwb_set_tile_shape", "uwb_tile_shape",
    "UwbError",
]

# UWB_LIBRARY=checked loads the bounds-checked build (build(checked=True))
_LIB_NAMES = {"": "libuwb.so", "checked": "libuwb_checked.so"}
if os.environ.get("UWB_LIBRARY", "") not in _LIB_NAMES:
    raise RuntimeError(f"UWB_LIBRARY={os.environ['UWB_LIBRARY']!r}: expected 'checked' or unset")
LIB_PATH = pathlib.Path(__file__).resolve().parent / _LIB_NAMES[os.environ.get("UWB_LIBRARY", "")]

UWB_OK = 0
UWB_ERR_ARG, UWB_ERR_CUDA, UWB_ERR_TIMEOUT = -1, -2, -3
UWB_ERR_NONFINITE, UWB_ERR_UNSUPPORTED, UWB_ERR_WORKSPACE = -4, -5, -6
UWB_ERR_BOUNDS = -7
UWB_DAS, UWB_DMAS, UWB_DMAS_LITERAL = 0, 1, 2
UWB_DECIM_MANUAL, UWB_DECIM_AUTO = 0, 1
UWB_METRIC_HYBRID, UWB_METRIC_MEAN, UWB_METRIC_VARIANCE, UWB_METRIC_HYBRID_UNCLIPPED = 0, 1, 2, 3
UWB_STOP_NONE, UWB_STOP_METRIC, UWB_STOP_MINSIZE, UWB_STOP_CAP, UWB_STOP_NO_TARGET = 0, 1, 2, 3, 4
UWB_MAX_ITERS = 32


class UwbError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed with status {code}: {uwb_last_error()}")
        self.code = code


class UwbGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("origin", ctypes.c_double * 3), ("pitch", ctypes.c_double * 3)]


class UwbRule(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("decimation", ctypes.c_int),
                ("min_tumor_diameter", ctypes.c_double), ("metric", ctypes.c_int),
                ("min_segment", ctypes.c_int), ("frame_num", ctypes.c_int),
                ("frame_den", ctypes.c_int), ("max_iters", ctypes.c_int)]


_I3 = ctypes.c_int * 3
_ITI = ctypes.c_int * UWB_MAX_ITERS
_IT3 = (ctypes.c_int * 3) * UWB_MAX_ITERS
_ITD = ctypes.c_double * UWB_MAX_ITERS


class UwbResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("n_logged", ctypes.c_int),
                ("stop_reason", ctypes.c_int), ("decim", ctypes.c_int), ("offset", _I3),
                ("dcount", _I3), ("roi_lo", _I3), ("roi_hi", _I3), ("loc_idx", _I3),
                ("points_evaluated", ctypes.c_longlong), ("loc_xyz", ctypes.c_double * 3),
                ("peak", ctypes.c_double), ("profile_max", ctypes.c_double),
                ("child", _ITI), ("n_children", _ITI), ("box_lo", _IT3), ("box_hi", _IT3),
                ("metric_top", _ITD), ("metric_gap", _ITD), ("between", _ITD),
                ("within", _ITD), ("stop_margin", _ITD)]


class UwbScan(ctypes.Structure):
    _fields_ = [("traces", ctypes.c_void_p), ("antennas", ctypes.c_void_p), ("M", ctypes.c_int),
                ("N", ctypes.c_int), ("grid", UwbGrid), ("v", ctypes.c_double),
                ("fs", ctypes.c_double)]


UWB_F32, UWB_F16, UWB_BF16 = 0, 1, 2

RESULT_DTYPE = np.dtype(UwbResult)
RESULT_BYTES = ctypes.sizeof(UwbResult)

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libuwb.so (built by ``paper_1709_02549_gb300.build.build()``)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(str(LIB_PATH))
        vp, i, ll, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double, \
            ctypes.c_size_t
        gp, rp = ctypes.POINTER(UwbGrid), ctypes.POINTER(UwbRule)
        sig = {
            "uwb_default_rule": (i, [rp]),
            "uwb_decimation": (i, [gp, rp]),
            "uwb_das_image": (i, [vp, i, i, vp, gp, d, d, i, vp, vp, vp]),
            "uwb_dmas_image": (i, [vp, i, i, vp, gp, d, d, i, i, vp, vp, vp]),
            "uwb_image_batch": (i, [i, i, vp, i, i, vp, ll, gp, d, d, i, vp, vp, vp]),
            "uwb_localize_workspace": (sz, [i, i, i, gp, i, rp]),
            "uwb_localize": (i, [vp, i, i, vp, gp, d, d, i, i, rp, vp, sz, vp, vp, vp]),
            "uwb_localize_batch": (i, [i, vp, i, i, vp, ll, gp, d, d, i, i, rp, vp, sz, vp, vp,
                                       vp]),
            "uwb_localize_batch_noalloc": (i, [i, vp, i, i, vp, ll, gp, d, d, i, i, rp, vp, vp,
                                               vp]),
            "uwb_localize_host_workspace": (sz, [i, vp, i, i, vp, ll, gp, d, d, i, i, rp]),
            "uwb_localize_host": (i, [i, vp, i, i, vp, ll, gp, d, d, i, i, rp, vp, sz, vp,
                                      ctypes.POINTER(ctypes.c_longlong), vp]),
            "uwb_presence_workspace": (sz, [i, i, i, gp, i, rp, i]),
            "uwb_presence_batch": (i, [i, vp, i, i, vp, ll, gp, d, d, i, i, rp, i, vp, sz, vp, vp,
                                       vp, vp]),
            "uwb_image_multistatic_batch": (i, [i, i, vp, i, i, vp, vp, i, ll, gp, d, d, i, vp, vp,
                                                vp]),
            "uwb_localize_multistatic_workspace": (sz, [i, i, i, gp, i, rp]),
            "uwb_localize_multistatic_batch": (i, [i, vp, i, i, vp, vp, i, ll, gp, d, d, i, i, rp,
                                                   vp, sz, vp, vp, vp]),
            "uwb_plan_create": (vp, [i, ctypes.POINTER(UwbScan), i, i, i, rp,
                                     ctypes.POINTER(ctypes.c_int)]),
            "uwb_plan_workspace": (sz, [vp]),
            "uwb_plan_image_offset": (ll, [vp, i]),
            "uwb_plan_upload": (i, [vp, vp, sz, vp]),
            "uwb_plan_images": (i, [vp, vp, vp, vp]),
            "uwb_plan_localize": (i, [vp, vp, vp]),
            "uwb_plan_destroy": (None, [vp]),
            "uwb_autotune": (i, [i, ctypes.POINTER(UwbScan), i, i, i, rp, vp, sz, vp,
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                  vp]),
            "uwb_set_tile_shape": (i, [i, i, ctypes.POINTER(ctypes.c_int)]),
            "uwb_tile_shape": (i, [i, i, ctypes.POINTER(ctypes.c_int)]),
            "uwb_device_status": (i, [i]),
            "uwb_phase_timing": (i, [i]),
            "uwb_phase_times": (i, [ctypes.POINTER(ctypes.c_double)]),
            "uwb_last_error": (ctypes.c_char_p, []),
            "uwb_measure_peaks": (i, [ctypes.POINTER(ctypes.c_double)] * 2),
            "uwb_wait_selftest": (i, [i]),
            "uwb_cnn_selftest": (i, [ctypes.POINTER(ctypes.c_int)]),
            "uwb_cnn_pack": (i, [vp, vp, vp]),
            "uwb_cnn_forward": (i, [vp, vp, i, vp, vp]),
            "uwb_cnn_train_workspace": (sz, [i]),
            "uwb_cnn_forward_record": (i, [vp, vp, vp, i, vp, vp, vp, sz, vp]),
            "uwb_cnn_gradients": (i, [vp, vp, vp, i, vp, vp, vp, sz, vp]),
            "uwb_cnn_adam": (i, [vp, vp, vp, vp, vp, i, ctypes.c_float, vp]),
            "uwb_cnn_train_step": (i, [vp, vp, vp, vp, vp, vp, i, i, ctypes.c_float, vp, vp, sz,
                                       vp]),
            "uwb_coarse_maps_workspace": (sz, [i]),
            "uwb_coarse_maps": (i, [i, vp, i, i, vp, ll, gp, d, d, i, vp, i, vp, vp, sz, vp]),
            "uwb_localize_progressive_workspace": (sz, [i, i, i, gp, i, rp]),
            "uwb_localize_progressive": (i, [i, vp, i, i, vp, ll, gp, d, d, i, i, rp, vp, sz, vp,
                                             vp]),
            "uwb_localize_learned_workspace": (sz, [i, gp, rp]),
            "uwb_localize_learned": (i, [i, vp, i, i, vp, ll, gp, d, d, i, i, rp, vp,
                                         ctypes.c_float, i, vp, sz, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def make_grid(grid) -> UwbGrid:
    if isinstance(grid, UwbGrid):
        return grid
    n = list(grid["n"]) + [1] * (3 - len(grid["n"]))
    origin = list(grid["origin"]) + [0.0] * (3 - len(grid["origin"]))
    pitch = list(grid["pitch"]) + [1.0] * (3 - len(grid["pitch"]))
    return UwbGrid(int(grid["dim"]), _I3(*n), (ctypes.c_double * 3)(*origin),
                   (ctypes.c_double * 3)(*pitch))


def uwb_last_error() -> str:
    return (lib().uwb_last_error() or b"").decode()


def _check(code: int, what: str) -> int:
    if code < 0:
        raise UwbError(code, what)
    return code


def _ptr(t, name: str, allow_none: bool = False):
    """Device address of a contiguous CUDA tensor (or None)."""
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _f32(t, name: str, allow_none: bool = False):
    import torch
    if t is not None and t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    return _ptr(t, name, allow_none)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def uwb_default_rule(**overrides) -> UwbRule:
    r = UwbRule()
    _check(lib().uwb_default_rule(ctypes.byref(r)), "uwb_default_rule")
    for k, v in overrides.items():
        setattr(r, k, v)
    return r


def uwb_decimation(grid, rule: UwbRule) -> int:
    return _check(lib().uwb_decimation(ctypes.byref(make_grid(grid)), ctypes.byref(rule)),
                  "uwb_decimation")


def uwb_das_image(traces, antennas, grid, v, fs, window, image, peak_index=None, stream=None):
    M, N = traces.shape[-2:]
    _check(lib().uwb_das_image(_f32(traces, "traces"), M, N, _f32(antennas, "antennas"),
                               ctypes.byref(make_grid(grid)), float(v), float(fs), int(window),
                               _f32(image, "image"), _ptr(peak_index, "peak_index", True),
                               _stream(stream)), "uwb_das_image")


def uwb_dmas_image(traces, antennas, grid, v, fs, window, literal_pairs, image, peak_index=None,
                   stream=None):
    M, N = traces.shape[-2:]
    _check(lib().uwb_dmas_image(_f32(traces, "traces"), M, N, _f32(antennas, "antennas"),
                                ctypes.byref(make_grid(grid)), float(v), float(fs), int(window),
                                int(bool(literal_pairs)), _f32(image, "image"),
                                _ptr(peak_index, "peak_index", True), _stream(stream)),
           "uwb_dmas_image")


def uwb_image_batch(beamformer, traces, antennas, grid, v, fs, window, image, peak_index=None,
                    stream=None):
    """traces [B, M, N]; antennas [M, 3] (shared) or [B, M, 3]; image [B, P]."""
    B, M, N = traces.shape
    stride = 0 if antennas.dim() == 2 else M * 3
    _check(lib().uwb_image_batch(B, int(beamformer), _f32(traces, "traces"), M, N,
                                 _f32(antennas, "antennas"), stride,
                                 ctypes.byref(make_grid(grid)), float(v), float(fs), int(window),
                                 _f32(image, "image"), _ptr(peak_index, "peak_index", True),
                                 _stream(stream)), "uwb_image_batch")


def uwb_localize_workspace(batch, M, N, grid, beamformer, rule: UwbRule) -> int:
    n = lib().uwb_localize_workspace(int(batch), int(M), int(N), ctypes.byref(make_grid(grid)),
                                     int(beamformer), ctypes.byref(rule))
    if n == 0:
        raise UwbError(UWB_ERR_ARG, "uwb_localize_workspace")
    return n


def uwb_localize(traces, antennas, grid, v, fs, window, beamformer, rule: UwbRule, workspace,
                 out, image=None, stream=None):
    """out: CUDA uint8 tensor of RESULT_BYTES bytes (device uwb_result)."""
    M, N = traces.shape[-2:]
    _check(lib().uwb_localize(_f32(traces, "traces"), M, N, _f32(antennas, "antennas"),
                              ctypes.byref(make_grid(grid)), float(v), float(fs), int(window),
                              int(beamformer), ctypes.byref(rule), _ptr(workspace, "workspace"),
                              workspace.numel() * workspace.element_size(), _ptr(out, "out"),
                              _f32(image, "image", True), _stream(stream)), "uwb_localize")


def uwb_localize_batch(traces, antennas, grid, v, fs, window, beamformer, rule: UwbRule,
                       workspace, out, image=None, stream=None):
    """traces [B, M, N]; antennas [M, 3] or [B, M, 3]; out uint8 [B * RESULT_BYTES]."""
    B, M, N = traces.shape
    stride = 0 if antennas.dim() == 2 else M * 3
    _check(lib().uwb_localize_batch(B, _f32(traces, "traces"), M, N, _f32(antennas, "antennas"),
                                    stride, ctypes.byref(make_grid(grid)), float(v), float(fs),
                                    int(window), int(beamformer), ctypes.byref(rule),
                                    _ptr(workspace, "workspace"),
                                    workspace.numel() * workspace.element_size(),
                                    _ptr(out, "out"), _f32(image, "image", True),
                                    _stream(stream)), "uwb_localize_batch")


def uwb_localize_progressive_workspace(batch, M, N, grid, beamformer, rule: UwbRule) -> int:
    n = lib().uwb_localize_progressive_workspace(int(batch), int(M), int(N),
                                                 ctypes.byref(make_grid(grid)), int(beamformer),
                                                 ctypes.byref(rule))
    if n == 0:
        raise UwbError(UWB_ERR_ARG, "uwb_localize_progressive_workspace")
    return n


def uwb_localize_progressive(traces, antennas, grid, v, fs, window, beamformer, rule: UwbRule,
                             workspace, out, stream=None):
    """Progressive re-evaluation; traces [B, M, N]; antennas [M, 3] or [B, M, 3];
    out uint8 [B * RESULT_BYTES]."""
    B, M, N = traces.shape
    stride = 0 if antennas.dim() == 2 else M * 3
    _check(lib().uwb_localize_progressive(B, _f32(traces, "traces"), M, N,
                                          _f32(antennas, "antennas"), stride,
                                          ctypes.byref(make_grid(grid)), float(v), float(fs),
                                          int(window), int(beamformer), ctypes.byref(rule),
                                          _ptr(workspace, "workspace"),
                                          workspace.numel() * workspace.element_size(),
                                          _ptr(out, "out"), _stream(stream)),
           "uwb_localize_progressive")


def _host_f32(a, name):
    import torch
    if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 host tensor")
    return ctypes.c_void_p(a.data_ptr())


def uwb_localize_host_workspace(traces_host, antennas_host, grid, v, fs, window, beamformer,
                                rule: UwbRule) -> int:
    B, M, N = traces_host.shape
    stride = 0 if antennas_host.dim() == 2 else M * 3
    n = lib().uwb_localize_host_workspace(B, _host_f32(traces_host, "traces"), M, N,
                                          _host_f32(antennas_host, "antennas"), stride,
                                          ctypes.byref(make_grid(grid)), float(v), float(fs),
                                          int(window), int(beamformer), ctypes.byref(rule))
    if n == 0:
        raise UwbError(UWB_ERR_ARG, "uwb_localize_host_workspace")
    return n


def uwb_localize_host(traces_host, antennas_host, grid, v, fs, window, beamformer, rule: UwbRule,
                      workspace, out_host, stream=None) -> int:
    """Host-memory localisation (traces [B, M, N] and antennas on the host, ideally
    pinned; out_host a host uint8 tensor of B * RESULT_BYTES). Returns the bytes
    copied host-to-device. Queued on the stream; synchronise before reading."""
    B, M, N = traces_host.shape
    stride = 0 if antennas_host.dim() == 2 else M * 3
    if out_host.is_cuda or out_host.numel() * out_host.element_size() < B * RESULT_BYTES:
        raise ValueError("out_host must be a host buffer of B * RESULT_BYTES bytes")
    moved = ctypes.c_longlong(0)
    _check(lib().uwb_localize_host(B, _host_f32(traces_host, "traces"), M, N,
                                   _host_f32(antennas_host, "antennas"), stride,
                                   ctypes.byref(make_grid(grid)), float(v), float(fs), int(window),
                                   int(beamformer), ctypes.byref(rule), _ptr(workspace, "workspace"),
                                   workspace.numel() * workspace.element_size(),
                                   ctypes.c_void_p(out_host.data_ptr()), ctypes.byref(moved),
                                   _stream(stream)), "uwb_localize_host")
    return int(moved.value)


def uwb_presence_workspace(batch, M, N, grid, beamformer, rule: UwbRule, decimation2) -> int:
    n = lib().uwb_presence_workspace(int(batch), int(M), int(N), ctypes.byref(make_grid(grid)),
                                     int(beamformer), ctypes.byref(rule), int(decimation2))
    if n == 0:
        raise UwbError(UWB_ERR_ARG, "uwb_presence_workspace")
    return n


def uwb_presence_batch(traces, antennas, grid, v, fs, window, beamformer, rule: UwbRule,
                       decimation2, workspace, out1, out2, present, stream=None):
    """Two-decimation tumour-presence test; present: int32 CUDA tensor [B]."""
    B, M, N = traces.shape
    stride = 0 if antennas.dim() == 2 else M * 3
    _check(lib().uwb_presence_batch(B, _f32(traces, "traces"), M, N, _f32(antennas, "antennas"),
                                    stride, ctypes.byref(make_grid(grid)), float(v), float(fs),
                                    int(window), int(beamformer), ctypes.byref(rule),
                                    int(decimation2), _ptr(workspace, "workspace"),
                                    workspace.numel() * workspace.element_size(),
                                    _ptr(out1, "out1"), _ptr(out2, "out2"),
                                    _ptr(present, "present"), _stream(stream)),
           "uwb_presence_batch")


def _i32(t, name):
    import torch
    if t.dtype != torch.int32:
        raise ValueError(f"{name} must be int32")
    return _ptr(t, name)


def uwb_image_multistatic_batch(beamformer, traces, channels, antennas, grid, v, fs, window,
                                image, peak_index=None, stream=None):
    """traces [B, C, N]; channels int32 [C, 2] (transmitter, receiver); antennas [M, 3]
    or [B, M, 3]; image [B, P]."""
    B, C, N = traces.shape
    M = antennas.shape[-2]
    stride = 0 if antennas.dim() == 2 else M * 3
    _check(lib().uwb_image_multistatic_batch(B, int(beamformer), _f32(traces, "traces"), C, N,
                                             _i32(channels, "channels"),
                                             _f32(antennas, "antennas"), M, stride,
                                             ctypes.byref(make_grid(grid)), float(v), float(fs),
                                             int(window), _f32(image, "image"),
                                             _ptr(peak_index, "peak_index", True),
                                             _stream(stream)), "uwb_image_multistatic_batch")


def uwb_localize_multistatic_workspace(batch, C, N, grid, beamformer, rule: UwbRule) -> int:
    n = lib().uwb_localize_multistatic_workspace(int(batch), int(C), int(N),
                                                 ctypes.byref(make_grid(grid)), int(beamformer),
                                                 ctypes.byref(rule))
    if n == 0:
        raise UwbError(UWB_ERR_ARG, "uwb_localize_multistatic_workspace")
    return n


def uwb_localize_multistatic_batch(traces, channels, antennas, grid, v, fs, window, beamformer,
                                   rule: UwbRule, workspace, out, image=None, stream=None):
    B, C, N = traces.shape
    M = antennas.shape[-2]
    stride = 0 if antennas.dim() == 2 else M * 3
    _check(lib().uwb_localize_multistatic_batch(B, _f32(traces, "traces"), C, N,
                                                _i32(channels, "channels"),
                                                _f32(antennas, "antennas"), M, stride,
                                                ctypes.byref(make_grid(grid)), float(v), float(fs),
                                                int(window), int(beamformer), ctypes.byref(rule),
                                                _ptr(workspace, "workspace"),
                                                workspace.numel() * workspace.element_size(),
                                                _ptr(out, "out"), _f32(image, "image", True),
                                                _stream(stream)), "uwb_localize_multistatic_batch")


class UwbPlan:
    """A ragged batch (scans of different antenna counts, trace lengths, grids):
    wraps uwb_plan_create / _upload / _images / _localize / _destroy. scans is a
    list of dicts {traces: CUDA tensor [M, N] (float32, float16 or bfloat16),
    antennas: CUDA float32 [M, 3], grid: dict, v, fs}; all traces share a dtype."""

    _DT = {"torch.float32": UWB_F32, "torch.float16": UWB_F16, "torch.bfloat16": UWB_BF16}

    def __init__(self, scans, window, beamformer, rule: UwbRule):
        self.B = len(scans)
        dts = {str(sc["traces"].dtype) for sc in scans}
        if len(dts) != 1 or next(iter(dts)) not in self._DT:
            raise ValueError("all traces must share one of float32/float16/bfloat16")
        self.dtype = self._DT[next(iter(dts))]
        self._keep = [(sc["traces"], sc["antennas"]) for sc in scans]
        arr = (UwbScan * self.B)()
        for k, sc in enumerate(scans):
            t, a = sc["traces"], sc["antennas"]
            if not (t.is_cuda and a.is_cuda and t.is_contiguous() and a.is_contiguous()):
                raise ValueError("traces and antennas must be contiguous CUDA tensors")
            arr[k] = UwbScan(t.data_ptr(), a.data_ptr(), int(t.shape[0]), int(t.shape[1]),
                             make_grid(sc["grid"]), float(sc["v"]), float(sc["fs"]))
        st = ctypes.c_int(0)
        self._arr, self._window, self._bf, self._rule = arr, int(window), int(beamformer), rule
        self.handle = lib().uwb_plan_create(self.B, arr, self.dtype, int(window), int(beamformer),
                                            ctypes.byref(rule), ctypes.byref(st))
        if not self.handle:
            raise UwbError(st.value, "uwb_plan_create")
        self.workspace = None

    def workspace_bytes(self) -> int:
        return lib().uwb_plan_workspace(self.handle)

    def image_offset(self, scan: int) -> int:
        return lib().uwb_plan_image_offset(self.handle, int(scan))

    def upload(self, workspace, stream=None):
        self.workspace = workspace
        _check(lib().uwb_plan_upload(self.handle, _ptr(workspace, "workspace"),
                                     workspace.numel() * workspace.element_size(),
                                     _stream(stream)), "uwb_plan_upload")

    def images(self, images, peak_index=None, stream=None):
        _check(lib().uwb_plan_images(self.handle, _f32(images, "images"),
                                     _ptr(peak_index, "peak_index", True), _stream(stream)),
               "uwb_plan_images")

    def localize(self, out, stream=None):
        _check(lib().uwb_plan_localize(self.handle, _ptr(out, "out"), _stream(stream)),
               "uwb_plan_localize")

    def autotune(self, workspace, out, stream=None):
        """Times the candidate tile shapes on this batch (uwb_autotune); returns
        (tile, ms). Later plans of the same beamformer/dimensionality use it."""
        tile = (ctypes.c_int * 3)()
        ms = ctypes.c_float(0)
        _check(lib().uwb_autotune(self.B, self._arr, self.dtype, self._window, self._bf,
                                  ctypes.byref(self._rule), _ptr(workspace, "workspace"),
                                  workspace.numel() * workspace.element_size(), _ptr(out, "out"),
                                  tile, ctypes.byref(ms), _stream(stream)), "uwb_autotune")
        return list(tile), ms.value

    def close(self):
        if getattr(self, "handle", None):
            lib().uwb_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_SCRATCH_BYTES = 16 << 20


def uwb_localize_batch_noalloc(traces, antennas, grid, v, fs, window, beamformer,
                               rule: UwbRule, out, image=None, stream=None):
    """uwb_localize_batch without a workspace: the library's built-in scratch
    (NOALLOC_SCRATCH_BYTES per device) is used instead, for callers that may not
    allocate device memory. Calls on one device must not overlap on the GPU."""
    B, M, N = traces.shape
    stride = 0 if antennas.dim() == 2 else M * 3
    _check(lib().uwb_localize_batch_noalloc(B, _f32(traces, "traces"), M, N,
                                            _f32(antennas, "antennas"), stride,
                                            ctypes.byref(make_grid(grid)), float(v), float(fs),
                                            int(window), int(beamformer), ctypes.byref(rule),
                                            _ptr(out, "out"), _f32(image, "image", True),
                                            _stream(stream)), "uwb_localize_batch_noalloc")


def uwb_phase_timing(enable: bool) -> None:
    _check(lib().uwb_phase_timing(int(bool(enable))), "uwb_phase_timing")


def uwb_phase_times():
    """(calls, [ms of phase 0..3]) summed since timing was switched on."""
    ms = (ctypes.c_double * 4)()
    calls = _check(lib().uwb_phase_times(ms), "uwb_phase_times")
    return calls, list(ms)


def uwb_set_tile_shape(beamformer, dim, tile=None) -> None:
    arr = None if tile is None else (ctypes.c_int * 3)(*tile)
    _check(lib().uwb_set_tile_shape(int(beamformer), int(dim), arr), "uwb_set_tile_shape")


def uwb_tile_shape(beamformer, dim):
    t = (ctypes.c_int * 3)()
    _check(lib().uwb_tile_shape(int(beamformer), int(dim), t), "uwb_tile_shape")
    return list(t)


def uwb_device_status(clear: bool = False) -> int:
    return lib().uwb_device_status(int(bool(clear)))


def results_from_device(out) -> np.ndarray:
    """Copies a device uwb_result array (uint8 tensor) to a numpy record array."""
    host = out.detach().to("cpu").numpy()
    return host.view(RESULT_DTYPE)


# ---------------------------------------------------------------- learned proposal
CNN_PARAMS = 18849
CNN_PACKED_BYTES = 38912
UWB_STOP_LEARNED = 5


def _nbytes(t):
    return t.numel() * t.element_size()


def uwb_cnn_selftest() -> bool:
    """Runs the tensor-core self-check on the current device (once)."""
    ok = ctypes.c_int(0)
    _check(lib().uwb_cnn_selftest(ctypes.byref(ok)), "uwb_cnn_selftest")
    return bool(ok.value)


def uwb_cnn_pack(theta, packed, stream=None):
    """theta: CUDA float32 [CNN_PARAMS]; packed: CUDA uint8 [CNN_PACKED_BYTES]."""
    _check(lib().uwb_cnn_pack(_f32(theta, "theta"), _ptr(packed, "packed"), _stream(stream)),
           "uwb_cnn_pack")


def uwb_cnn_forward(packed, maps, scores, stream=None):
    """maps: CUDA float32 [B, 32, 32]; scores: CUDA float32 [B, 16]."""
    _check(lib().uwb_cnn_forward(_ptr(packed, "packed"), _f32(maps, "maps"), maps.shape[0],
                                 _f32(scores, "scores"), _stream(stream)), "uwb_cnn_forward")


CNN_RECORD_BYTES = 242688


def uwb_cnn_forward_record(packed, maps, scores, record, labels=None, loss=None, stream=None):
    """uwb_cnn_forward that also fills `record` (CUDA uint8 [B * CNN_RECORD_BYTES]);
    with labels (CUDA int32 [B]) also dz and the loss (CUDA float32 [1])."""
    _check(lib().uwb_cnn_forward_record(_ptr(packed, "packed"), _f32(maps, "maps"),
                                        _ptr(labels, "labels", True), maps.shape[0],
                                        _f32(scores, "scores"), _ptr(loss, "loss", True),
                                        _ptr(record, "record"),
                                        record.numel() * record.element_size(),
                                        _stream(stream)), "uwb_cnn_forward_record")


def cnn_record_arrays(record, B: int) -> dict:
    """Decodes B maps' forward records (host bytes, the layout of
    UWB_CNN_RECORD_BYTES in uwb.h) into float64 arrays: X0 [B, 32, 32], A1, A2,
    A3 [B, 32, 32, 32] (channel first), F [B, 16, 32], dz [B, 16]."""
    raw = np.asarray(record, dtype=np.uint8)[:B * CNN_RECORD_BYTES].reshape(B, CNN_RECORD_BYTES)
    y, x = np.mgrid[0:32, 0:32]
    u = 34 + 33 * y + x                                         # [32, 32]
    x0 = raw[:, :5120].copy().view(np.float32)                  # [B, 1280]
    out = {"X0": x0[:, u].astype(np.float64)}
    c = np.arange(32)[:, None, None]
    off = (c // 8) * 19616 + 16 * u[None] + 2 * (c % 8)         # [32, 32, 32]
    for name, base in (("A1", 5120), ("A2", 83584), ("A3", 162048)):
        lo = raw[:, base + off].astype(np.uint32)
        hi = raw[:, base + off + 1].astype(np.uint32)
        bits = ((hi << 8) | lo) << 16
        out[name] = bits.view(np.float32).astype(np.float64)
    out["F"] = raw[:, 240512:240512 + 2048].copy().view(np.float32).reshape(B, 16, 32) \
        .astype(np.float64)
    out["dz"] = raw[:, 242560:242560 + 64].copy().view(np.float32).astype(np.float64)
    return out


def uwb_cnn_train_workspace(batch) -> int:
    n = lib().uwb_cnn_train_workspace(int(batch))
    if n == 0:
        raise UwbError(UWB_ERR_ARG, "uwb_cnn_train_workspace")
    return n


def uwb_cnn_gradients(packed, maps, labels, grad, loss, workspace, stream=None):
    """labels: CUDA int32 [B]; grad: CUDA float32 [CNN_PARAMS]; loss: CUDA float32 [1]."""
    _check(lib().uwb_cnn_gradients(_ptr(packed, "packed"), _f32(maps, "maps"),
                                   _i32(labels, "labels"), maps.shape[0], _f32(grad, "grad"),
                                   _f32(loss, "loss"), _ptr(workspace, "workspace"),
                                   _nbytes(workspace), _stream(stream)), "uwb_cnn_gradients")


def uwb_cnn_adam(theta, m, v, grad, packed, step, lr, stream=None):
    _check(lib().uwb_cnn_adam(_f32(theta, "theta"), _f32(m, "m"), _f32(v, "v"),
                              _f32(grad, "grad"), _ptr(packed, "packed"), int(step), float(lr),
                              _stream(stream)), "uwb_cnn_adam")


def uwb_cnn_train_step(theta, m, v, packed, maps, labels, step, lr, loss, workspace, stream=None):
    _check(lib().uwb_cnn_train_step(_f32(theta, "theta"), _f32(m, "m"), _f32(v, "v"),
                                    _ptr(packed, "packed"), _f32(maps, "maps"),
                                    _i32(labels, "labels"), maps.shape[0], int(step), float(lr),
                                    _f32(loss, "loss"), _ptr(workspace, "workspace"),
                                    _nbytes(workspace), _stream(stream)), "uwb_cnn_train_step")


def uwb_coarse_maps_workspace(batch) -> int:
    return lib().uwb_coarse_maps_workspace(int(batch))


def uwb_coarse_maps(traces, antennas, grid, v, fs, window, side, maps, region_lo=None,
                    workspace=None, stream=None):
    """traces [B, M, N]; antennas [M, 3] or [B, M, 3]; maps CUDA float32 [B, 32, 32];
    region_lo: CUDA int32 [B, 2] (x, y) or None (the region at the origin)."""
    B, M, N = traces.shape
    stride = 0 if antennas.dim() == 2 else M * 3
    _check(lib().uwb_coarse_maps(B, _f32(traces, "traces"), M, N, _f32(antennas, "antennas"),
                                 stride, ctypes.byref(make_grid(grid)), float(v), float(fs),
                                 int(window), None if region_lo is None else
                                 _i32(region_lo, "region_lo"), int(side), _f32(maps, "maps"),
                                 _ptr(workspace, "workspace", True),
                                 0 if workspace is None else _nbytes(workspace),
                                 _stream(stream)), "uwb_coarse_maps")


def uwb_localize_learned_workspace(batch, grid, rule: UwbRule) -> int:
    n = lib().uwb_localize_learned_workspace(int(batch), ctypes.byref(make_grid(grid)),
                                             ctypes.byref(rule))
    if n == 0:
        raise UwbError(UWB_ERR_ARG, "uwb_localize_learned_workspace")
    return n


def uwb_localize_learned(traces, antennas, grid, v, fs, window, beamformer, rule: UwbRule, packed,
                         threshold, levels, workspace, out, stream=None):
    """traces [B, M, N]; antennas [M, 3] or [B, M, 3]; out uint8 [B * RESULT_BYTES]."""
    B, M, N = traces.shape
    stride = 0 if antennas.dim() == 2 else M * 3
    _check(lib().uwb_localize_learned(B, _f32(traces, "traces"), M, N, _f32(antennas, "antennas"),
                                      stride, ctypes.byref(make_grid(grid)), float(v), float(fs),
                                      int(window), int(beamformer), ctypes.byref(rule),
                                      _ptr(packed, "packed"), float(threshold), int(levels),
                                      _ptr(workspace, "workspace"), _nbytes(workspace),
                                      _ptr(out, "out"), _stream(stream)), "uwb_localize_learned")


def uwb_wait_selftest(probes: int) -> None:
    """Bounded-wait self-check: a wait that nothing completes runs out after
    `probes` probes and records UWB_ERR_TIMEOUT in the device status word."""
    _check(lib().uwb_wait_selftest(int(probes)), "uwb_wait_selftest")


def uwb_measure_peaks():
    """(FP32 TFLOP/s of paired-FMA chains, conflict-free shared-load wavefronts/s)."""
    t, w = ctypes.c_double(), ctypes.c_double()
    _check(lib().uwb_measure_peaks(ctypes.byref(t), ctypes.byref(w)), "uwb_measure_peaks")
    return t.value, w.value

