"""Builds ``librecon.so`` in-tree for sm_103a: nvcc for the kernels, g++ for the host
plan (with ``-ffp-contract=off`` so the FP64 plan constants follow the written
operation order on every host), compiled in parallel and linked with the static
CUDA runtime.  ``python -m paper_2206_09151_gb300.build`` or ``build()``."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librecon.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU_SOURCES = ["stage_a.cu", "backproject.cu", "backproject_tma.cu", "density.cu", "learned.cu", "noalloc.cu", "fft3.cu", "fourier.cu"]
CPP_SOURCES = ["plan.cpp"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _sources_newer_than(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "recon.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra_nvcc: list[str] | None = None) -> str:
    """Compiles every source and links ``librecon.so``; returns its path."""
    if not force and not _sources_newer_than(LIB):
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-I" + os.path.join(cuda, "include")]
    os.makedirs(OUT_DIR, exist_ok=True)
    jobs = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"] + inc + \
              (extra_nvcc or []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((src, cmd))
        objs.append(obj)
    for src in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall"] + inc + \
              ["-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((src, cmd))
        objs.append(obj)
    procs = [(name, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
             for name, cmd in jobs]
    failed = []
    logs = {}
    for name, cmd, pr in procs:
        out, _ = pr.communicate()
        logs[name] = out
        if pr.returncode != 0:
            failed.append((name, cmd, out))
    with open(os.path.join(OUT_DIR, "ptxas.log"), "w") as f:
        for name, out in logs.items():
            f.write(f"== {name}\n{out}\n")
    if failed:
        msg = "\n".join(f"[{n}] {' '.join(c)}\n{o}" for n, c, o in failed)
        raise RuntimeError("librecon build failed:\n" + msg)
    if verbose:
        for name, out in logs.items():
            print(f"== {name}\n{out}")
    tmp = LIB + ".tmp"
    link = [nvcc, ARCH, "-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("librecon link failed:\n" + " ".join(link) + "\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
