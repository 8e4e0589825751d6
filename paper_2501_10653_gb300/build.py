"""Build ``libiqa.so`` (the C-ABI library of ``include/iqa.h``) in-tree for sm_103a.

Every ``csrc/*.cu`` and ``csrc/*.cpp`` is compiled by nvcc in parallel with
``-gencode arch=compute_103a,code=sm_103a`` and linked into
``paper_2501_10653_gb300/libiqa.so``.  A content hash of the sources, headers
and flags skips the build when nothing changed.  ``build(checked=True)`` makes
the bounds-checked variant ``libiqa_checked.so`` (``-DIQA_CHECKS=1``: every
kernel checks the geometry of its accesses and counts failures, see
``iqa_debug_violations``) for the tests; the product library has no checks.
"""
import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(ROOT, "_build", "libiqa")
LIB = os.path.join(PKG, "libiqa.so")
BUILD_DIR_CHECKED = os.path.join(ROOT, "_build", "libiqa_checked")
LIB_CHECKED = os.path.join(PKG, "libiqa_checked.so")
CHECK_FLAGS = ["-DIQA_CHECKS=1"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-O2", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"),
                 "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libiqa")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) +
                  glob.glob(os.path.join(CSRC, "*.cpp")))


def _digest(extra=()):
    h = hashlib.sha256()
    files = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) +
                                glob.glob(os.path.join(CSRC, "*.cuh")) +
                                glob.glob(os.path.join(INCLUDE, "*.h")))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + list(extra)).encode())
    return h.hexdigest()


def _compile(nvcc, src, extra_flags, verbose, build_dir=BUILD_DIR):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [nvcc] + NVCC_FLAGS + extra_flags + ["-c", src, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc] + NVCC_FLAGS + extra_flags + ["-x", "cu", "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or r.returncode != 0:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s" % os.path.basename(src))
    return obj


def build(force=False, verbose=False, ptxas_info=False, jobs=None, checked=False):
    """Compile and link libiqa.so (libiqa_checked.so with checked=True);
    returns its path."""
    build_dir = BUILD_DIR_CHECKED if checked else BUILD_DIR
    lib = LIB_CHECKED if checked else LIB
    defs = CHECK_FLAGS if checked else []
    stamp = os.path.join(build_dir, "stamp")
    digest = _digest(defs)
    if (not force and os.path.exists(lib) and os.path.exists(stamp)
            and open(stamp).read() == digest):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    extra = defs + (["-Xptxas", "-v"] if ptxas_info else [])
    srcs = _sources()
    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, extra, verbose or ptxas_info,
                                              build_dir), srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(digest)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                ptxas_info="--ptxas" in sys.argv))
