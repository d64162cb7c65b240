"""Build libaimx.so in-tree with nvcc for sm_103a (no CMake, parallel per-file compiles)."""

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libaimx.so")
SOURCES = ["setup.cu", "fft.cu", "matvec.cu", "fused.cu", "solve.cu", "precond.cu", "gnn.cu", "batch.cu", "ports.cu",
           "aim.cu", "tune.cu", "noalloc.cu", "peak.cu", "charge.cu", "sweep.cu", "api.cu"]
HEADERS = ["aimx_internal.h", "cplx.cuh", "fftreg.cuh", "regfft.cuh", "geom.cuh", "krylov.cuh"]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-diag-suppress", "177"]
# extra nvcc flags and an output directory for side-by-side builds (e.g. AIMX_NVCC_FLAGS="-DNAME")
EXTRA = os.environ.get("AIMX_NVCC_FLAGS", "").split()
if os.environ.get("AIMX_LIB_DIR"):
    OUT_DIR = os.environ["AIMX_LIB_DIR"]
    LIB = os.path.join(OUT_DIR, "libaimx.so")


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libaimx")
    return p


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _newest_input():
    files = [os.path.join(CSRC, s) for s in _sources()]
    files += [os.path.join(CSRC, h) for h in HEADERS if os.path.exists(os.path.join(CSRC, h))]
    files.append(os.path.join(os.path.dirname(HERE), "include", "aimx.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force=False, verbose=False):
    """Compile every translation unit (in parallel) and link libaimx.so; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(os.path.dirname(HERE), "include")]

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc] + GENCODE + FLAGS + EXTRA + inc + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = _sources()
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + GENCODE + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lcufft"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
