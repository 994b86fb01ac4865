"""The benchmark's reference arm (the FP64 oracle on the host) prints the
contract's JSON line; runs on CPU."""
import json
import subprocess
import sys

from conftest import ROOT


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                        "--config", "das2d_64", "--steps", "2", "--warmup", "3",
                        "--cpu-pool", "2"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "scans/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_kernel_hash_follows_code_not_comments():
    """The ncu traffic figures are keyed to a hash of the kernel code: comment
    and blank-line edits keep it, any code edit changes it, and comment
    markers inside string literals are code."""
    sys.path.insert(0, str(ROOT))
    import bench
    src = 'int f(int a) {  // add one\n  /* body */\n  return a + 1;\n}\n\nconst char* s = "x//y";\n'
    same = ('/* header */\nint f(int a) {\n\n  return a + 1;  // one more\n}\n'
            'const char* s = "x//y";')
    assert bench.code_only(src) == bench.code_only(same)
    assert bench.code_only(src) != bench.code_only(src.replace("a + 1", "a + 2"))
    assert '"x//y"' in bench.code_only(src)
    assert len(bench.kernel_sha()) == 16


def test_image_roofline_takes_the_resource_with_the_larger_demand():
    """DAS and identity-DMAS bench lines: the operation count per focal point by
    hand, and the binding resource chosen by demand per point (shared-load
    wavefronts M (W + 1) / 32 against FP32-pipe operations / 128)."""
    sys.path.insert(0, str(ROOT))
    import bench
    # DAS, M = 32, W = 20: per antenna 3 + 3 + 1 + 1 (delay) + 1 (1 - f) + 40;
    # per point 20 energy multiply-adds
    assert bench.fp32_ops_per_point(0, 32, 20) == 32 * 49 + 20 == 1588
    # identity DMAS: per antenna 8 + 4 x 20, per point 4 x 20
    assert bench.fp32_ops_per_point(1, 32, 20) == 32 * 88 + 80 == 2896
    # multistatic, 12 antennas and 144 channels: 6 per antenna, 3 + 80 per channel
    assert bench.fp32_ops_per_point(1, 12, 20, channels=144) == 72 + 144 * 83 + 80
    n_pts, ms = 1.0e6, 2.0
    das = bench.load_or_alu_roofline(n_pts, 32, 20, 1588.0, ms, 312e9, 78.0)
    idm = bench.load_or_alu_roofline(n_pts, 32, 20, 2896.0, ms, 312e9, 78.0)
    assert das["bound"] == "smem" and das["other_resource"]["name"] == "alu"
    assert idm["bound"] == "alu" and idm["other_resource"]["name"] == "smem"
    wf = n_pts * 32 * 21 / 32
    assert das["wavefronts_per_launch"] == idm["wavefronts_per_launch"] == wf
    assert abs(das["achieved"] - wf / 2e-3 / 1e9) < 1e-9
    assert abs(das["frac"] - das["achieved"] / bench.LDS_PEAK_GWF) < 1e-12
    assert abs(idm["achieved"] - n_pts * 2896 / 2e-3 / 1e12) < 1e-12
    assert abs(idm["frac"] - idm["achieved"] / bench.FP32_PIPE_PEAK_TOPS) < 1e-12
    # the measured FP32 ceiling is quoted in TFLOP/s: a multiply-add is 2 FLOP, 1 operation
    assert abs(idm["measured_peak"] - 39.0) < 1e-12
    # both resources are reported whichever binds
    assert abs(idm["other_resource"]["frac"] - das["frac"]) < 1e-12


def test_flop_count_per_point():
    """Algorithmic FLOP per focal point: 10 + 2W per antenna, plus W M(M - 1)
    for literal DMAS pairs or W (2M + 3) for the identity form. At 32 antennas
    and W = 20 the literal count is 21 440; a full 512^2 literal image is then
    5.6e9 FLOP and a 256^3 one with 64 antennas 1.4e12."""
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.flops_per_point(2, 32, 20) == 32 * 50 + 20 * 32 * 31 == 21440
    assert bench.flops_per_point(1, 32, 20) == 32 * 50 + 20 * 67
    assert bench.flops_per_point(0, 32, 20) == 32 * 50
    assert round(512 ** 2 * bench.flops_per_point(2, 32, 20) / 1e9, 1) == 5.6
    assert round(256 ** 3 * bench.flops_per_point(2, 64, 20) / 1e12, 1) == 1.4


def test_derived_peaks_follow_the_device():
    sys.path.insert(0, str(ROOT))
    import bench
    old = (bench.SMS, bench.SM_MAX_GHZ)
    try:
        bench.configure_peaks(148, 1.98)
        assert abs(bench.FP32_PEAK_TFLOPS - 148 * 128 * 2 * 1.98 / 1e3) < 1e-9
        assert abs(bench.LDS_PEAK_GWF - 148 * 1.98) < 1e-9
        assert abs(bench.FP32_PIPE_PEAK_TOPS - 148 * 128 * 1.98 / 1e3) < 1e-9
        assert "148 SMs" in bench.peak_source("flops")
    finally:
        bench.configure_peaks(*old)
