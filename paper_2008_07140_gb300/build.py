"""Build libqsim.so in-tree: nvcc for sm_103a, one object per translation unit, in parallel."""

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqsim.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["api.cpp", "gates.cpp", "planner.cpp", "tune.cpp", "diag.cpp", "sweep.cu", "reduce.cu", "remap.cu",
           "fused_simt.cu", "fused_tc.cu", "noalloc.cu", "df.cu", "traj.cu",
           "partial.cu"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The split complex128 kernels are error-free transformations (TwoSum, TwoProduct): a
# product contracted into a following addition would break them, so in df.cu only the
# explicit fmaf calls are fused.
EXTRA = {"df.cu": ["-fmad=false"]}
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
          "--expt-relaxed-constexpr"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libqsim)")


def _deps_mtime():
    newest = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            newest = max(newest, os.path.getmtime(os.path.join(d, f)))
    return max(newest, os.path.getmtime(__file__))


def up_to_date():
    return os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime()


def _compile(src, verbose):
    obj = os.path.join(BUILD, src + ".o")
    cmd = [nvcc()] + ARCH + COMMON
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    cmd += EXTRA.get(src, [])
    cmd += ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False):
    """Compile every CUDA/C++ source and link libqsim.so next to this file."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    workers = min(len(SOURCES), os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if verbose:
        for (_, log), src in zip(results, SOURCES):
            if log.strip():
                sys.stderr.write("== %s\n%s" % (src, log))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
