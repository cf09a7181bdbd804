"""Build libpch.so in-tree with nvcc for sm_103a (no cmake, one -gencode, parallel TUs)."""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpch.so")
SOURCES = ["mesh.cu", "radix.cu", "solver.cu", "controller.cu", "contour.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "--expt-relaxed-constexpr"]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cuda, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build_id(files) -> str:
    """First 16 hex digits of the SHA-256 of the library's sources: compiled in as
    PCH_BUILD_ID, it keys the autotuner's cache so that timings taken with other kernels
    are never reused."""
    h = hashlib.sha256()
    for f in sorted(files):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "pch.h"))
    bid = build_id(headers + [os.path.join(CSRC, s) for s in SOURCES])
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        # the autotuner (solver.cu) carries the build id of every source
        deps = [s] + headers + ([os.path.join(CSRC, x) for x in SOURCES] if src == "solver.cu" else [])
        if force or _stale(o, deps):
            jobs.append([_nvcc(), *NVCC_FLAGS, f"-DPCH_BUILD_ID=\"{bid}\"", "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", LIB, *objs, "-lcudart_static",
             "-Xcompiler", "-fPIC"])
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
