"""Build libgks.so (CUDA, sm_103a) in-tree.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2309_10534_gb300/libgks.so``.  Objects go to ``_build/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
OUT = os.path.join(HERE, "libgks.so")
ROOT = os.path.dirname(HERE)

UNITS = ["gks_api", "gks_k1d", "gks_k2d_f32", "gks_k2d_f64", "gks_opcount", "gks_host_replica", "gks_noalloc", "gks_probe", "gks_ensemble", "gks_adjoint", "gks_flips"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
          "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _sources():
    inc = os.path.join(ROOT, "include")
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(inc, f) for f in os.listdir(inc)]


# float32 device arithmetic: flush denormals, approximate divide and square
# root (these flags do not touch float64 operations)
FAST_F32 = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]
# (the adjoint recomputes the forward pass's float32 selections and
# reconstructions, so it takes the same flags as the forward kernels)
EXTRA = {"gks_k2d_f32": FAST_F32, "gks_k1d": FAST_F32, "gks_ensemble": FAST_F32, "gks_adjoint": FAST_F32,
         "gks_flips": FAST_F32}


def _compile(unit):
    src = os.path.join(CSRC, unit + ".cu")
    obj = os.path.join(BUILD, unit + ".o")
    log = os.path.join(BUILD, unit + ".log")
    cmd = [_nvcc()] + ARCH + COMMON + EXTRA.get(unit, []) + ["-c", src, "-o", obj]
    with open(log, "w") as f:
        r = subprocess.run(cmd, stdout=f, stderr=subprocess.STDOUT)
    if r.returncode:
        with open(log) as f:
            sys.stderr.write(f.read())
        raise RuntimeError("nvcc failed for %s" % unit)
    return obj


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(p) for p in _sources())
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= newest:
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(_compile, UNITS))
    tmp = OUT + ".tmp%d" % os.getpid()
    subprocess.run([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-ldl"], check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
