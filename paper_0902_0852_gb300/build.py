"""Build libhk.so (the CUDA library behind the C ABI in include/hk.h) in-tree.

Compiles every translation unit in csrc/ for sm_103a only, in parallel, then
links a shared library next to this file.  Objects go to _build/ (ignored by
git).  Rebuilds only when a source or header is newer than the library.

``build(checked=True)`` makes libhk_checked.so instead: the same code with
the device-side bounds checks on (HK_CHECKED) and a synchronisation after
every launch that names the launch behind a fault or a failed check.  The
binding loads it when the environment sets HK_CHECKED=1.  It is a diagnosis
build, far slower than libhk.so.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhk.so")
LIB_CHECKED = os.path.join(HERE, "libhk_checked.so")
SOURCES = ["hk_api.cu", "hk_update.cu", "hk_panel.cu", "hk_solve.cu", "hk_selftest.cu", "hk_peaks.cu", "hk_update_i8.cu", "hk_batch.cu", "hk_mlp.cu", "hk_ldlt.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhk")
    return path


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "hk.h"))
    return files


def needs_build(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force=False, verbose=False, extra=(), checked=False):
    """Compile and link libhk.so (or libhk_checked.so); returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not needs_build(lib):
        return lib
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    flags = FLAGS + (["-DHK_CHECKED"] if checked else [])

    def one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc] + flags + list(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
