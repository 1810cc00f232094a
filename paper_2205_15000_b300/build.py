"""Build the C-ABI library libsc.so (CUDA for sm_103a) in-tree.

    python -m paper_2205_15000_b300.build
"""
import concurrent.futures
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libsc.so")
# the same sources with every table index checked in the kernels (-DSC_DEBUG_BOUNDS)
LIB_CHECKED = os.path.join(LIBDIR, "libsc_checked.so")
SOURCES = ["kernels.cu", "sweep_f32.cu", "sweep_side_f32.cu", "sweep_f64.cu", "lattice_f32.cu", "adjoint.cu", "adjoint_f32.cu",
           "adjoint_f64.cu", "api.cpp", "batch.cpp", "geometry.cpp", "noalloc.cu", "accel.cu", "accel_api.cpp", "ozaki.cpp", "vecpot.cu"]
HEADERS = ["bounds.cuh", "kernels.cuh", "sweep_kernel.cuh", "geometry.hpp", "riccati_step.cuh", "context.hpp", "adjoint.cuh",
           "adjoint_kernel.cuh", "adjoint_x2.cuh", "accel.cuh", "vecpot.cuh", "sweep_x2.cuh", "lattice_f32.cuh"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "sc.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, obj, verbose, checked=False):
    cmd = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
    if checked:
        cmd.insert(1, "-DSC_DEBUG_BOUNDS")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), flush=True)
    return subprocess.run(cmd, capture_output=not verbose, text=True)


def build(force=False, verbose=False, checked=False):
    """Compile every source to an object (in parallel) and link libsc.so, or,
    with checked=True, the bounds-checked libsc_checked.so."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    objdir = os.path.join(LIBDIR, "obj_checked" if checked else "obj")
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, f + ".o") for f in SOURCES]
    workers = max(1, min(len(SOURCES), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda so: _compile(so[0], so[1], verbose, checked), zip(SOURCES, objs)))
    for src, r in zip(SOURCES, results):
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout or ''}{r.stderr or ''}")
    link = [NVCC, *ARCH, "-shared", "-o", lib + ".tmp", *objs, "-lcudart"]
    subprocess.run(link, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
