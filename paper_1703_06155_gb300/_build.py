"""Compile libh2.so (all of csrc/) and the peak probes libh2peaks.so
(peaks/) for sm_103a with nvcc, in place.

Translation units are compiled in parallel and only when a source or header
changed; objects go to paper_1703_06155_gb300/_build/ (git-ignored).
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libh2.so")
PEAKS_SRC = os.path.join(PKG, "peaks", "peaks.cu")
PEAKS_LIB = os.path.join(PKG, "libh2peaks.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC,
         "--expt-relaxed-constexpr", "-diag-suppress", "177"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libh2)")


def _headers_mtime():
    hs = (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
          + glob.glob(os.path.join(INCLUDE, "*.h")))
    return max(os.path.getmtime(h) for h in hs)


def build(force=False, verbose=False, jobs=None):
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hmt = _headers_mtime()

    def compile_one(src):
        obj = os.path.join(OBJ, os.path.basename(src) + ".o")
        if (not force and os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(src)
                and os.path.getmtime(obj) >= hmt):
            return obj, None
        cmd = [nvcc] + ARCH + FLAGS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            return obj, "%s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr)
        if verbose:
            sys.stdout.write(r.stdout + r.stderr)
        return obj, None

    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        res = list(ex.map(compile_one, srcs))
    errs = [e for _, e in res if e]
    if errs:
        raise RuntimeError("libh2 compilation failed:\n" + "\n".join(errs))
    objs = [o for o, _ in res]
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("libh2 link failed:\n%s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, LIB)
    # arithmetic peak probes (measurement only; not part of libh2)
    if force or not os.path.exists(PEAKS_LIB) or os.path.getmtime(PEAKS_SRC) > os.path.getmtime(PEAKS_LIB):
        tmp = PEAKS_LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-O3", "-shared", "-Xcompiler", "-fPIC", "-o", tmp, PEAKS_SRC]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("libh2peaks build failed:\n%s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, PEAKS_LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
