"""Build libisingfilm.so in-tree: nvcc for the sm_103a kernels, g++ for the host C ABI.

    python -m paper_1205_5588_gb300.build        # or build() from Python

Translation units compile in parallel; the CUDA runtime is linked statically so the library
works next to whatever runtime PyTorch brought.  Host code is built with -ffp-contract=off so
the fp64 threshold tables round the same way on x86-64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libisingfilm.so"
LIB_PATH = os.path.join(OUT_DIR, LIB_NAME)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels_sweep.cu", "kernels_words.cu", "kernels_slabs.cu", "kernels_resident.cu", "kernels_aux.cu",
              "noalloc.cu", "kernels_peak.cu"]
CPP_SOURCES = ["capi.cpp", "batch.cpp", "serve.cpp", "lattice.cpp", "schedule.cpp"]
HEADERS = ["isf_internal.h", "device_common.cuh", "sweep_core.cuh", "grid_sync.cuh", "capi_internal.h", "trace.h"]


def cuda_home() -> str:
    for k in ("CUDA_HOME", "CUDA_PATH"):
        if os.environ.get(k):
            return os.environ[k]
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _sources():
    inc = os.path.join(os.path.dirname(HERE), "include")
    return [os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES + HEADERS] + [
        os.path.join(inc, "isingfilm.h"), os.path.join(inc, "isingfilm_tuning.h")]


def is_stale(path: str = LIB_PATH) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, extra_nvcc=()) -> str:
    """Compile every CUDA/C++ source for sm_103a and link libisingfilm.so; returns its path."""
    if not force and not is_stale():
        return LIB_PATH
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    os.makedirs(OUT_DIR, exist_ok=True)
    inc = ["-I", os.path.join(home, "include"), "-I", CSRC]
    jobs = []
    for s in CU_SOURCES:
        o = os.path.join(OUT_DIR, s + ".o")
        jobs.append(([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                      "-Xptxas", "-v" if verbose else "-O3", *extra_nvcc, *inc, "-c",
                      os.path.join(CSRC, s), "-o", o], o))
    for s in CPP_SOURCES:
        o = os.path.join(OUT_DIR, s + ".o")
        jobs.append((["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", *inc, "-c",
                      os.path.join(CSRC, s), "-o", o], o))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        logs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for l in logs:
            sys.stderr.write(l)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    _run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *[o for _, o in jobs], "-lpthread", "-ldl"])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
