"""In-tree build of the native libraries (no cmake, no pip install).

    lib/libfrgen.so     seeded input generators (gcc)
    lib/libflowref.so   the CUDA path behind include/flowref.h (nvcc, sm_103a only)

Translation units compile in parallel; the CUDA library takes one -gencode
(compute_103a -> sm_103a).  Host code is compiled with -ffp-contract=off so that
the budget expression floor((1 + alpha*eps) * W / k) is evaluated without fused
multiply-adds on both x86-64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(HERE, "lib", "obj")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")

CUDA_SOURCES = [
    "api.cu",
    "api_batch.cu",
    "api_active.cu",
    "api_mt.cu",
    "api_ml.cu",
    "fm_kernel.cu",
    "mt_kernel.cu",
    "ml_kernel.cu",
    "round_kernel.cu",
    "prep_kernel.cu",
    "serve.cu",
    "noalloc.cu",
    "cluster_flow.cu",
    "queue_sweep.cu",
    "api_queue.cu",
]


def _nvcc():
    p = os.path.join(CUDA_HOME, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _stale(out, srcs):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(s) > t for s in srcs)


def build_inputs(force=False):
    os.makedirs(LIBDIR, exist_ok=True)
    src = os.path.join(CSRC, "inputs", "frgen.c")
    out = os.path.join(LIBDIR, "libfrgen.so")
    if force or _stale(out, [src]):
        _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", out, src, "-lm"])
    return out


def _headers():
    hs = [os.path.join(ROOT, "include", "flowref.h")]
    for d, _, fs in os.walk(CSRC):
        hs += [os.path.join(d, f) for f in fs if f.endswith((".cuh", ".h"))]
    return hs


def build_cuda(force=False, verbose=False, extra=()):
    os.makedirs(OBJDIR, exist_ok=True)
    out = os.path.join(LIBDIR, "libflowref.so")
    srcs = [os.path.join(CSRC, s) for s in CUDA_SOURCES]
    deps = srcs + _headers()
    if not force and not _stale(out, deps):
        return out
    common = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]
    if verbose:
        common += ["-Xptxas", "-v"]

    def one(src):
        obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
        log = _run(common + ["-rdc=false", "-c", src, "-o", obj])
        return obj, log

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        res = list(ex.map(one, srcs))
    objs = [o for o, _ in res]
    _run([_nvcc(), *ARCH, "-shared", "-o", out, *objs, "-lcudart", "-lpthread"])
    if verbose:
        for _, log in res:
            sys.stdout.write(log)
    return out


def build_all(force=False, verbose=False):
    a = build_inputs(force)
    b = build_cuda(force, verbose)
    return a, b


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv, verbose="-v" in sys.argv))
