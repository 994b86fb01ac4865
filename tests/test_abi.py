"""The C ABI library on the host: it loads, exports every declared entry point,
and rejects bad arguments before touching the GPU (no compute calls here)."""
import ctypes
import re

import pytest

from conftest import ROOT


def declared_functions():
    text = (ROOT / "include" / "uwb.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(uwb_[a-z_]+)\s*\(", text)))


def test_every_declared_function_is_exported(uwb):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(uwb.lib(), name), name


def test_structure_sizes_match_the_header(uwb):
    # uwb_result: 20 ints, 1 int64, 5 doubles, 256 ints of logs, 160 doubles
    assert uwb.RESULT_BYTES == 20 * 4 + 8 + 5 * 8 + 256 * 4 + 5 * 32 * 8
    assert ctypes.sizeof(uwb.UwbGrid) == 4 + 12 + 48
    assert ctypes.sizeof(uwb.UwbRule) == 4 + 4 + 8 + 4 * 4 + 4 + 4


def test_default_rule(uwb):
    r = uwb.uwb_default_rule()
    assert (r.mode, r.metric, r.min_segment, r.frame_num, r.frame_den, r.max_iters) == \
        (uwb.UWB_DECIM_AUTO, uwb.UWB_METRIC_HYBRID, 4, 1, 4, 0)
    assert r.min_tumor_diameter == pytest.approx(0.01)


def test_automatic_decimation_worked_example(uwb):
    # Section IV: 1 cm tumour at 1 mm resolution -> 7
    grid = {"dim": 2, "n": [100, 100, 1], "origin": [0, 0, 0], "pitch": [1e-3, 1e-3, 1.0]}
    assert uwb.uwb_decimation(grid, uwb.uwb_default_rule()) == 7
    g512 = {"dim": 2, "n": [512, 512, 1], "origin": [0, 0, 0], "pitch": [0.12 / 512] * 2 + [1.0]}
    assert uwb.uwb_decimation(g512, uwb.uwb_default_rule()) == 30
    manual = uwb.uwb_default_rule(mode=uwb.UWB_DECIM_MANUAL, decimation=5)
    assert uwb.uwb_decimation(grid, manual) == 5


def test_workspace_grows_with_the_batch(uwb):
    g = {"dim": 2, "n": [512, 512, 1], "origin": [0, 0, 0], "pitch": [0.12 / 512] * 2 + [1.0]}
    r = uwb.uwb_default_rule()
    one = uwb.uwb_localize_workspace(1, 32, 2048, g, uwb.UWB_DMAS_LITERAL, r)
    many = uwb.uwb_localize_workspace(64, 32, 2048, g, uwb.UWB_DMAS_LITERAL, r)
    assert 0 < one < many
    assert many >= 64 * 18 * 18 * 4      # the decimated profiles


@pytest.mark.parametrize("kw,code", [
    ({"M": 0}, -1), ({"N": 0}, -1), ({"window": 0}, -1), ({"v": 0.0}, -1),
    ({"fs": float("nan")}, -1), ({"dim": 4}, -1), ({"n2": 3}, -1), ({"pitch": 0.0}, -1),
    ({"null_traces": True}, -1),
])
def test_bad_arguments_are_rejected_on_the_host(uwb, kw, code):
    L = uwb.lib()
    g = uwb.make_grid({"dim": kw.get("dim", 2), "n": [8, 8, kw.get("n2", 1)],
                       "origin": [0, 0, 0], "pitch": [kw.get("pitch", 1e-3)] * 2 + [1.0]})
    fake = ctypes.c_void_p(0x1000)           # never dereferenced: checks come first
    tr = None if kw.get("null_traces") else fake
    st = L.uwb_das_image(tr, kw.get("M", 4), kw.get("N", 64), fake, ctypes.byref(g),
                         kw.get("v", 1e8), kw.get("fs", 5e10), kw.get("window", 4), fake, None,
                         None)
    assert st == code
    assert uwb.uwb_last_error() != ""


def test_bad_rule_and_workspace_are_rejected(uwb):
    L = uwb.lib()
    g = uwb.make_grid({"dim": 2, "n": [8, 8, 1], "origin": [0, 0, 0], "pitch": [1e-3] * 2 + [1.0]})
    fake = ctypes.c_void_p(0x1000)
    bad = uwb.uwb_default_rule(metric=9)
    assert L.uwb_localize(fake, 4, 64, fake, ctypes.byref(g), 1e8, 5e10, 4, uwb.UWB_DAS,
                          ctypes.byref(bad), fake, 1 << 20, fake, None, None) == -1
    ok = uwb.uwb_default_rule()
    assert L.uwb_localize(fake, 4, 64, fake, ctypes.byref(g), 1e8, 5e10, 4, uwb.UWB_DAS,
                          ctypes.byref(ok), None, 0, fake, None, None) == -6
    assert L.uwb_localize(fake, 4, 64, fake, ctypes.byref(g), 1e8, 5e10, 4, uwb.UWB_DAS,
                          ctypes.byref(ok), ctypes.c_void_p(0x1008), 1 << 20, fake, None,
                          None) == -6
    assert L.uwb_localize(fake, 4, 64, fake, ctypes.byref(g), 1e8, 5e10, 4, 7,
                          ctypes.byref(ok), fake, 1 << 20, fake, None, None) == -1
    # literal pairs are built for up to 96 antennas
    assert L.uwb_dmas_image(fake, 97, 64, fake, ctypes.byref(g), 1e8, 5e10, 4, 1, fake, None,
                            None) == -5


def test_tile_shape_table(uwb):
    # linear tiles by default, reported as {0, 0, 0}
    assert uwb.uwb_tile_shape(uwb.UWB_DAS, 2) == [0, 0, 0]
    assert uwb.uwb_tile_shape(uwb.UWB_DMAS_LITERAL, 3) == [0, 0, 0]
    uwb.uwb_set_tile_shape(uwb.UWB_DAS, 2, [16, 16, 1])
    assert uwb.uwb_tile_shape(uwb.UWB_DAS, 2) == [16, 16, 1]
    uwb.uwb_set_tile_shape(uwb.UWB_DAS, 2, [0, 0, 0])
    assert uwb.uwb_tile_shape(uwb.UWB_DAS, 2) == [0, 0, 0]
    uwb.uwb_set_tile_shape(uwb.UWB_DMAS_LITERAL, 3, [8, 4, 4])
    assert uwb.uwb_tile_shape(uwb.UWB_DMAS_LITERAL, 3) == [8, 4, 4]
    uwb.uwb_set_tile_shape(uwb.UWB_DMAS_LITERAL, 3, None)
    assert uwb.uwb_tile_shape(uwb.UWB_DMAS_LITERAL, 3) == [0, 0, 0]
    for bad in ([16, 8, 1], [24, 8, 1], [16, 4, 4]):   # wrong size, not a power of 2, z in 2-D
        with pytest.raises(uwb.UwbError):
            uwb.uwb_set_tile_shape(uwb.UWB_DAS, 2, bad)


def test_learned_proposal_arguments_are_rejected_on_the_host(uwb):
    L = uwb.lib()
    fake = ctypes.c_void_p(0x1000)
    ok = uwb.uwb_default_rule()
    sq = uwb.make_grid({"dim": 2, "n": [512, 512, 1], "origin": [0, 0, 0],
                        "pitch": [2e-4] * 2 + [1.0]})
    rect = uwb.make_grid({"dim": 2, "n": [512, 256, 1], "origin": [0, 0, 0],
                          "pitch": [2e-4] * 2 + [1.0]})
    odd = uwb.make_grid({"dim": 2, "n": [96, 96, 1], "origin": [0, 0, 0],
                         "pitch": [2e-4] * 2 + [1.0]})

    def learned(grid, threshold=0.5, levels=2, ws=fake, nbytes=1 << 30):
        return L.uwb_localize_learned(4, fake, 8, 256, fake, 0, ctypes.byref(grid), 1e8, 5e10, 4,
                                      uwb.UWB_DAS, ctypes.byref(ok), fake, threshold, levels, ws,
                                      nbytes, fake, None)

    assert learned(rect) == uwb.UWB_ERR_UNSUPPORTED          # not square
    assert learned(odd, levels=2) == uwb.UWB_ERR_UNSUPPORTED  # two levels need a multiple of 128
    assert learned(sq, levels=4) == uwb.UWB_ERR_ARG
    assert learned(sq, threshold=1.5) == uwb.UWB_ERR_ARG
    assert learned(sq, ws=None) == uwb.UWB_ERR_WORKSPACE
    assert learned(sq, nbytes=16) == uwb.UWB_ERR_WORKSPACE
    assert uwb.uwb_localize_learned_workspace(4, sq, ok) > 4 * 32 * 32 * 4
    assert L.uwb_cnn_train_workspace(0) == 0
    assert L.uwb_cnn_train_workspace(8) >= 8 * 242688 + 4 * uwb.CNN_PARAMS
    assert L.uwb_cnn_forward(fake, fake, 0, fake, None) == uwb.UWB_ERR_ARG
    assert L.uwb_cnn_adam(fake, fake, fake, fake, fake, 0, 1e-3, None) == uwb.UWB_ERR_ARG
    assert L.uwb_cnn_adam(fake, fake, fake, fake, fake, 1, -1.0, None) == uwb.UWB_ERR_ARG
    assert L.uwb_cnn_gradients(fake, fake, fake, 4, fake, fake, None, 0, None) == \
        uwb.UWB_ERR_WORKSPACE
    # coarse maps: the side must be a multiple of 32 inside the grid
    assert L.uwb_coarse_maps(4, fake, 8, 256, fake, 0, ctypes.byref(sq), 1e8, 5e10, 4, None, 48,
                             fake, None, 0, None) == uwb.UWB_ERR_ARG
    assert L.uwb_coarse_maps(4, fake, 8, 256, fake, 0, ctypes.byref(sq), 1e8, 5e10, 4, fake, 64,
                             fake, None, 0, None) == uwb.UWB_ERR_WORKSPACE


def test_wait_selftest_rejects_probe_counts_on_the_host(uwb):
    L = uwb.lib()
    for probes in (0, -5, (1 << 24) + 1):
        assert L.uwb_wait_selftest(probes) == uwb.UWB_ERR_ARG
        assert "probes" in uwb.uwb_last_error()


def _header_define(name):
    text = (ROOT / "include" / "uwb.h").read_text()
    m = re.search(r"#define\s+" + name + r"\s+(.+)", text)
    assert m, name
    value = re.sub(r"/\*.*", "", m.group(1)).strip()  # a trailing comment
    return eval(re.sub(r"(\d+)u\b", r"\1", value))


def test_binding_constants_equal_the_header(uwb):
    assert uwb.NOALLOC_SCRATCH_BYTES == _header_define("UWB_NOALLOC_SCRATCH_BYTES")
    assert uwb.CNN_RECORD_BYTES == _header_define("UWB_CNN_RECORD_BYTES")
    assert uwb.CNN_PARAMS == _header_define("UWB_CNN_PARAMS")
    assert uwb.CNN_PACKED_BYTES == _header_define("UWB_CNN_PACKED_BYTES")
    for name in ("UWB_OK", "UWB_ERR_ARG", "UWB_ERR_CUDA", "UWB_ERR_TIMEOUT", "UWB_ERR_NONFINITE",
                 "UWB_ERR_UNSUPPORTED", "UWB_ERR_WORKSPACE", "UWB_ERR_BOUNDS"):
        assert getattr(uwb, name) == _header_define(name), name
