"""Build ``libdg.so`` (the C-ABI library of ``include/dg.h``) in-tree with nvcc.

Every translation unit is compiled for sm_103a only, in parallel, then linked
into ``paper_1305_5536_gb300/libdg.so``.  Rebuilds only what changed.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdg.so")
SOURCES = ["dg_capi.cu", "dg_misc.cu", "dg_k2d.cu", "dg_k3d.cu", "dg_k3m.cu", "dg_kmh.cu", "dg_kmh3d.cu",
           "dg_kmh3m.cu", "dg_adjoint.cu",
           "dg_noalloc.cu", "dg_batch.cu", "dg_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps_mtime():
    t = 0.0
    for f in os.listdir(CSRC):
        t = max(t, os.path.getmtime(os.path.join(CSRC, f)))
    t = max(t, os.path.getmtime(os.path.join(ROOT, "include", "dg.h")))
    return t


# Forward stage kernels: FP32 division and square root to within 2 ulp (the
# single-precision path only; double precision is always IEEE-exact).
FAST_FP32 = ["-prec-div=false", "-prec-sqrt=false"]
FAST_FP32_SOURCES = ("dg_k2d.cu", "dg_k3d.cu", "dg_k3m.cu", "dg_kmh.cu", "dg_kmh3d.cu", "dg_kmh3m.cu",
                     "dg_batch.cu")


def _compile(src, extra, obj=OBJ):
    out = os.path.join(obj, src.replace(".cu", ".o"))
    fast = FAST_FP32 if src in FAST_FP32_SOURCES else []
    cmd = [_nvcc()] + ARCH + FLAGS + fast + extra + ["-c", os.path.join(CSRC, src), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return out, r.stderr


# The phase-profiling build: the same sources with clock64() stamps between the
# stage kernels' phases (DG_PHASE_PROFILE), in a library of its own.
PHASE_OBJ = os.path.join(PKG, "_build_phase")
PHASE_LIB = os.path.join(PKG, "libdg_phase.so")


def build(force=False, verbose=False, extra=(), phase=False):
    obj, lib = (PHASE_OBJ, PHASE_LIB) if phase else (OBJ, LIB)
    if phase:
        extra = tuple(extra) + ("-DDG_PHASE_PROFILE",)
    os.makedirs(obj, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    extra = list(extra)
    if verbose:
        extra += ["-Xptxas", "-v"]
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, obj), SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                phase="--phase" in sys.argv))
