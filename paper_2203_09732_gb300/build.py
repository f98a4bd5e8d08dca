"""Builds libhs.so (the C ABI of include/hs.h) in-tree with nvcc for sm_103a.

    python -m paper_2203_09732_gb300.build        # or build() from Python

Translation units compile in parallel; the shared library is relinked only
when a source or header is newer than it.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUTDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUTDIR, "libhs.so")
SOURCES = ["api.cu", "hv.cu", "minres.cu", "vec.cu", "twist.cu", "lanczos.cu", "twist_noalloc.cu", "hv_sb.cu", "minres_sb.cu", "observables.cu", "adjoint.cu", "minres_pipe.cu", "sweep.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(HERE, "..", "include", "hs.h"))
    return hdrs


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, extra=(), lib=None, objdir=None):
    lib = lib or LIB
    objdir = objdir or OBJDIR
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    os.makedirs(objdir, exist_ok=True)
    hdrs = _deps()
    cc = nvcc()
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(objdir, s.replace(".cu", ".o"))
        if _newer(obj, [src] + hdrs):
            jobs.append([cc, *FLAGS, *extra, "-c", src, "-o", obj])
    objs = [os.path.join(objdir, s.replace(".cu", ".o")) for s in SOURCES]

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        list(ex.map(run, jobs))
    if jobs or _newer(lib, objs):
        run([cc, *ARCH, "-shared", "-o", lib, *objs, "-lcudart"])
    return lib


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
    print(LIB)
