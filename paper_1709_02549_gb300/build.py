"""Builds libuwb.so in-tree with nvcc for sm_103a (translation units in parallel).

build(checked=True) builds libuwb_checked.so beside it, compiled with
-DUWB_CHECK: the image kernels check every staged-window run, image index and
profile index they compute and record UWB_ERR_BOUNDS instead of leaving their
buffers (the package loads it when UWB_LIBRARY=checked)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import pathlib
import shutil
import subprocess

PKG = pathlib.Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = ROOT / "_build"
LIB = PKG / "libuwb.so"
BUILD_CHECKED = ROOT / "_build_checked"
LIB_CHECKED = PKG / "libuwb_checked.so"
SOURCES = ["uwb_api.cu", "select_kernels.cu", "image_das.cu", "image_dmas.cu",
           "image_literal.cu", "cnn.cu", "peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}",
                f"-I{CSRC}"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newest_input() -> float:
    files = list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h"))
    files.append(pathlib.Path(__file__))
    return max(f.stat().st_mtime for f in files)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> pathlib.Path:
    lib, build_dir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    flags = FLAGS + (["-DUWB_CHECK"] if checked else [])
    if lib.exists() and not force and lib.stat().st_mtime >= _newest_input():
        return lib
    nvcc = _nvcc()
    build_dir.mkdir(exist_ok=True)

    def compile_one(src: str) -> pathlib.Path:
        obj = build_dir / (src.replace(".cu", ".o"))
        cmd = [nvcc, *flags, "-c", str(CSRC / src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib.with_suffix(f".so.{os.getpid()}.tmp")
    cmd = [nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
