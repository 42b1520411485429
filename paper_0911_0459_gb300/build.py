"""Build the CUDA library in-tree: paper_0911_0459_gb300/_lib/liblbgb300.so (sm_103a).

Each translation unit under csrc/ is compiled by its own nvcc process, in
parallel, then linked into one shared library with the C ABI of include/lb.h.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT, "liblbgb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return exe


def cuda_libdir():
    base = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for d in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        if os.path.isdir(os.path.join(base, d)):
            return os.path.join(base, d)
    return "/usr/local/cuda/lib64"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), variant: str = "") -> str:
    """Compile and link the library; variant="check" builds the bounds-checked debug
    library (-DLB_CHECK) into _lib/check/ instead."""
    out_dir, lib = OUT, LIB
    if variant == "check":
        out_dir = os.path.join(OUT, "check")
        lib = os.path.join(out_dir, "liblbgb300.so")
        extra = ("-DLB_CHECK", *extra)
    elif variant:
        raise ValueError(f"unknown variant {variant!r}")
    os.makedirs(out_dir, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    flags = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
             "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([nvcc(), *flags, "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, res):
            if verbose or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or not os.path.exists(lib):
        libdir = cuda_libdir()
        cmd = [nvcc(), "-shared", *ARCH, "-o", lib + ".tmp", *objs, "-cudart", "shared",
               "-L", libdir, "-Xlinker", "-rpath=" + libdir]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force="--force" in sys.argv, verbose=v or bool(extra), extra=extra,
                variant="check" if "--check" in sys.argv else ""))
