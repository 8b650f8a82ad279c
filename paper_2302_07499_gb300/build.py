"""In-tree build of libnlfem.so for sm_103a (nvcc, one -gencode, parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnlfem.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

# translation units compiled without fused multiply-add: the FP64 decisions of
# the method follow a fixed operation order there
NO_FMA = {"nl_pairs.cu", "nl_assemble64.cu"}
SOURCES = ["nl_util.cu", "nl_pairs.cu", "nl_assemble64.cu", "nl_assemble32.cu", "nl_reduce.cu",
           "nl_api.cu", "nl_solve.cu", "nl_probe.cu", "nl_batch.cu", "nl_server.cu", "nl_peaks.cu"]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
          "-I", CSRC]


def _deps_mtime():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "nlfem.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _compile(src, verbose=False):
    obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
    cmd = [NVCC] + GENCODE + COMMON + (["-fmad=false"] if src in NO_FMA else []) + \
        (["-Xptxas", "-v"] if verbose else []) + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    with cf.ThreadPoolExecutor(max_workers=min(8, len(SOURCES))) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if verbose:
        for _, err in results:
            sys.stderr.write(err)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + GENCODE + ["-shared", "-cudart", "static", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
