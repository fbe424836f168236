"""Build ``libnslct.so`` in-tree with nvcc for sm_103a (GB300).

Every translation unit compiles in parallel; unchanged objects are reused.
Run ``python -m paper_1707_03688_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(PKG, "libnslct.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC] + ARCH
# extra nvcc flags (e.g. -DNSLCT_E_LARGE=16 to build the radix-16 variant of the 2048/4096 kernels)
EXTRA = os.environ.get("NSLCT_NVCC_FLAGS", "").split()


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libnslct")


def _units():
    """(source, object, extra flags) for every translation unit."""
    units = []
    for real, tag in (("float", "f32"), ("double", "f64")):
        for g in range(4):
            defs = [f"-DNSLCT_REAL={real}", f"-DNSLCT_GROUP={g}", f"-DNSLCT_SUFFIX={tag}_g{g}"]
            units.append(("passes.cu", f"passes_{tag}_g{g}.o", defs))
    for src in sorted(os.listdir(CSRC)):
        if src == "passes.cu":
            continue
        if src.endswith(".cu") or src.endswith(".cpp"):
            units.append((src, os.path.splitext(src)[0] + ".o", []))
    return units


def _deps_mtime() -> float:
    newest = 0.0
    stamp = os.path.join(BUILD_DIR, "flags.txt")
    flags = " ".join(EXTRA)
    if not os.path.exists(stamp) or open(stamp).read() != flags:
        os.makedirs(BUILD_DIR, exist_ok=True)
        with open(stamp, "w") as f:
            f.write(flags)
    newest = max(newest, os.path.getmtime(stamp))
    for d in (CSRC, INCLUDE):
        for name in os.listdir(d):
            newest = max(newest, os.path.getmtime(os.path.join(d, name)))
    newest = max(newest, os.path.getmtime(os.path.abspath(__file__)))
    return newest


def build(verbose: bool = False, jobs: int | None = None, force: bool = False) -> str:
    """Compile and link libnslct.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    deps = _deps_mtime()
    units = _units()

    def compile_one(unit):
        src, obj, extra = unit
        obj_path = os.path.join(BUILD_DIR, obj)
        if not force and os.path.exists(obj_path) and os.path.getmtime(obj_path) >= deps:
            return obj_path, None
        cmd = [nvcc] + COMMON + EXTRA + extra + ["-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj_path]
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            return obj_path, res.stdout + res.stderr
        return obj_path, None

    workers = jobs or min(len(units), max(2, os.cpu_count() or 2))
    with ThreadPoolExecutor(max_workers=workers) as pool:
        results = list(pool.map(compile_one, units))
    errors = [err for _, err in results if err]
    if errors:
        raise RuntimeError("libnslct build failed:\n" + "\n".join(errors))
    objs = [path for path, _ in results]
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc, "-shared", "-cudart", "static"] + ARCH + objs + ["-o", LIB_PATH]
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("libnslct link failed:\n" + res.stdout + res.stderr)
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
