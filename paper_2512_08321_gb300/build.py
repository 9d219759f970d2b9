"""Build the CUDA library in-tree: paper_2512_08321_gb300/libozaki2emu.so, and
the cuBLAS interposer libozaki2emu_preload.so.

Every translation unit under csrc/ is compiled for sm_103a only (one
-gencode), in parallel, then linked against the shared CUDA runtime so the
library and PyTorch share one runtime and one primary context.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "libozaki2emu.so")
PRELOAD = os.path.join(HERE, "libozaki2emu_preload.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
              "--expt-relaxed-constexpr", "-I", os.path.join(os.path.dirname(HERE), "include")]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _compile(src, nvcc, extra):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-x", "cu", "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, extra=()):
    """Compile and link; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    srcs = sources()
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, nvcc, list(extra)), srcs))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    build_preload(nvcc)
    return LIB


def build_preload(nvcc=None):
    """The LD_PRELOAD interposer (host code only): libozaki2emu_preload.so beside
    the library, linked to it with an $ORIGIN run path; cuBLAS is not linked
    (its routines are looked up at run time in the libraries loaded after it)."""
    nvcc = nvcc or _nvcc()
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        raise RuntimeError("g++ not found")
    tmp = PRELOAD + ".tmp"
    cmd = [cxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, os.path.join(HERE, "preload", "ozaki2_preload.cpp"),
           "-I", os.path.join(os.path.dirname(HERE), "include"), "-I", os.path.join(cuda, "include"),
           "-L", HERE, "-lozaki2emu", "-L", os.path.join(cuda, "lib64"), "-lcudart", "-ldl",
           "-Wl,-rpath,$ORIGIN"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"preload build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PRELOAD)
    return PRELOAD


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
