"""Build ``librbm.so`` (the C-ABI library of ``include/rbm.h``) in-tree.

Each translation unit is compiled by nvcc for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``) in parallel, then linked into
``paper_1812_10575_gb300/_build/librbm.so`` with the static CUDA runtime.
No PyTorch types cross the boundary, so no torch extension machinery is used.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, extra defines) per object
UNITS = [
    ("rbm_abi.cu", []),
    ("perm_step.cu", []),
    ("rec_step.cu", []),
    ("direct.cu", ["-DRBM_DIRECT_F32"]),
    ("direct.cu", ["-DRBM_DIRECT_F64"]),
    ("noalloc.cu", []),
    ("coop_step.cu", []),
    ("batched.cu", []),
    ("surrogate.cu", []),
    ("rbmr.cu", []),
    ("peak.cu", []),
]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return path


def _sources():
    out = []
    for root, _, files in os.walk(CSRC):
        out += [os.path.join(root, f) for f in files if f.endswith((".cu", ".cuh", ".h"))]
    out.append(os.path.join(ROOT, "include", "rbm.h"))
    return out


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources()) or os.path.getmtime(__file__) > t


def _compile(src: str, defs: list[str], obj: str, verbose_ptxas: bool) -> None:
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
           "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), *defs, "-c",
           os.path.join(CSRC, src), "-o", obj]
    if verbose_ptxas:
        cmd.insert(1, "-Xptxas=-v")
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src} {defs}:\n{p.stderr}")
    if verbose_ptxas:
        with open(obj + ".ptxas.txt", "w") as f:
            f.write(p.stderr)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile (if stale) and return the path of ``librbm.so``."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs = []
    jobs = []
    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        for src, defs in UNITS:
            tag = src.replace(".cu", "") + "".join(d.replace("-D", "_").lower() for d in defs)
            obj = os.path.join(BUILD, tag + ".o")
            objs.append(obj)
            jobs.append(ex.submit(_compile, src, defs, obj, verbose_ptxas))
        for j in jobs:
            j.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n" + p.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv))
