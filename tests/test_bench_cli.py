"""The benchmark's reference arm (the FP64 oracle on the host) prints the
contract's JSON line; runs on CPU."""
import json
import subprocess
import sys

from conftest import ROOT


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                        "--config", "das2d_64", "--steps", "2", "--warmup", "3",
                        "--ref-scans-per-step", "1"], capture_output=True, text=True,
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
