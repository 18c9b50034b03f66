"""Build the hn CUDA library (libhn.so) in-tree for sm_103a with nvcc, and its checked variant
libhn_debug.so (the same sources with HN_DEBUG_CHECKS=1: index checks in the kernels, guard bytes
around device blocks; see include/hn_debug.h).

Each translation unit compiles in parallel to an object file under _build/ (_build/debug/ for the
checked variant), then the objects are linked into ``paper_0904_4152_gb300/libhn.so`` and
``libhn_debug.so``.  Only one ``-gencode`` target (sm_103a) is built.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libhn.so")
LIB_DEBUG = os.path.join(HERE, "libhn_debug.so")
SOURCES = ["k_cycle.cu", "k_setup.cu", "engine.cu", "api.cu", "serve.cu", "noalloc.cu", "blas1.cu",
           "band4.cu", "peaks.cu", "tune_cache.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhn.so")
    return cand


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    return max(os.path.getmtime(f) for f in files)


def _link(objs, lib):
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libhn.so and the checked variant libhn_debug.so (HN_DEBUG_CHECKS=1), all translation
    units of both compiled in one pool; returns the path of libhn.so."""
    deps = _deps()
    todo = [(lib, dbg) for lib, dbg in ((LIB, False), (LIB_DEBUG, True))
            if force or not os.path.exists(lib) or os.path.getmtime(lib) < deps]
    if not todo:
        return LIB
    nvcc = _nvcc()

    def compile_one(job):
        src, dbg = job
        out_dir = os.path.join(BUILD, "debug") if dbg else BUILD
        os.makedirs(out_dir, exist_ok=True)
        obj = os.path.join(out_dir, src + ".o")
        cmd = [nvcc, *ARCH, *FLAGS] + (["-DHN_DEBUG_CHECKS=1"] if dbg else []) + \
              ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    jobs = [(src, dbg) for _, dbg in todo for src in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), max(4, os.cpu_count() or 4))) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    k = 0
    for lib, _ in todo:
        _link([o for o, _ in results[k:k + len(SOURCES)]], lib)
        k += len(SOURCES)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
