"""Build libtsvd.so in-tree with nvcc for sm_103a (GB300).

Each .cu file is compiled to an object in parallel, then linked into
paper_2603_11953_gb300/_build/libtsvd.so (static CUDA runtime), and the peak
probe (peak_probe.cu) into _build/libtsvd_probe.so.  Run as
``python -m paper_2603_11953_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libtsvd.so")
PROBE_LIB = os.path.join(OUT, "libtsvd_probe.so")
PROBE_SOURCE = "peak_probe.cu"
SOURCES = ["tsvd_api.cu", "gram_ozaki.cu", "jacobi.cu", "compute_u.cu", "compute_u_tc.cu", "gram_static.cu", "eig_onesided.cu", "tma_util.cu", "gram_tc.cu", "gram_fp64.cu", "eig_dd.cu", "batch.cu", "eig_alg2.cu", "gram_sharded.cu", "cholqr.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                "-Xcompiler", "-fvisibility=hidden", "-I", os.path.join(HERE, "..", "include")]


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC] + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(OUT, exist_ok=True)
    extra = extra or []
    srcs = [os.path.join(CSRC, s) for s in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "tsvd.h")]
    if not force and os.path.exists(LIB) and os.path.exists(PROBE_LIB):
        newest = max(os.path.getmtime(s) for s in srcs)
        if min(os.path.getmtime(LIB), os.path.getmtime(PROBE_LIB)) >= newest:
            return LIB
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES + [PROBE_SOURCE]))
    for lib, parts in ((LIB, objs[:-1]), (PROBE_LIB, objs[-1:])):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + parts
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None))
