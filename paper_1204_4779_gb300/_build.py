"""Build libhydro.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel into ``_build/``; the shared library lands next to
this file.  FP64 translation units use ``--fmad=false`` (one correctly rounded IEEE operation
per arithmetic operation); FP32 ones keep FMA contraction and flush denormals.

    python -m paper_1204_4779_gb300._build [--force] [--verbose]
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhydro.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# translation unit -> extra flags
UNITS = {
    "stage_f32_d3.cu": ["-ftz=true"],
    "stage_f32_d3b.cu": ["-ftz=true"],
    "stage_f32_d12.cu": ["-ftz=true"],
    "stage_f64.cu": ["--fmad=false"],
    "aux_kernels.cu": ["--fmad=false"],
    "hydro_abi.cu": [],
    "static_step.cu": [],
    "batch_f32.cu": ["-ftz=true"],
    "batch_f64.cu": ["--fmad=false"],
    "batch_abi.cu": [],
    "mlp.cu": [],
    "wave.cu": ["--fmad=false"],
    "diag.cu": [],
    "analytic.cu": ["--fmad=false"],
    "exchange.cu": [],
    "tma_host.cu": [],
}
HEADERS = ["hydro_device.cuh", "stage_kernel.cuh", "stage_launch.cuh", "hydro_internal.h",
           "batch_kernel.cuh", "tma.cuh"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhydro.so")


def _base_flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC] + ARCH


def _digest(unit: str, flags) -> str:
    h = hashlib.sha256()
    for name in [unit] + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    with open(os.path.join(ROOT, "include", "hydro.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(flags).encode())
    return h.hexdigest()[:16]


def _compile(unit: str, force: bool, verbose: bool) -> str:
    flags = _base_flags() + UNITS[unit]
    tag = _digest(unit, flags)
    obj = os.path.join(OUT_DIR, f"{os.path.splitext(unit)[0]}.{tag}.o")
    if os.path.exists(obj) and not force:
        return obj
    cmd = [nvcc(), "-c", os.path.join(CSRC, unit), "-o", obj + ".tmp"] + flags
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr[-6000:]}")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libhydro.so; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(u, force, verbose), UNITS))
    # objects of earlier sources or flags are never linked again: drop them
    keep = {os.path.basename(o) for o in objs}
    for name in os.listdir(OUT_DIR):
        if name.endswith(".o") and name not in keep:
            try:
                os.remove(os.path.join(OUT_DIR, name))
            except OSError:
                pass
    stamp = os.path.join(OUT_DIR, "lib.stamp")
    key = "|".join(objs)
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == key:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(key)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
