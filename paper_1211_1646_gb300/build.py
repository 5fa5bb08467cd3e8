"""Build libhdmc.so (the CUDA library behind include/hdmc.h) for sm_103a.

Each .cu file is compiled to an object in parallel, then linked into
paper_1211_1646_gb300/_build/libhdmc.so.  Device code is compiled with
-fmad=false and host code with -ffp-contract=off: results must not depend
on which multiply-adds the compiler would fuse.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libhdmc.so")
# the bounds-checked debug build (-DHDMC_CHECK), kept apart from the product
CHECK_DIR = os.path.join(HERE, "_build_check")
CHECK_LIB = os.path.join(CHECK_DIR, "libhdmc.so")
SOURCES = ["hdmc_api.cu", "hdmc_host.cu", "hdmc_batch.cu", "hdmc_draws.cu", "hdmc_f32.cu", "hdmc_f64.cu",
           "hdmc_noalloc.cu", "hdmc3.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "-I" + INCLUDE, "-I" + CSRC]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhdmc.so")
    return exe


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "hdmc.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force=False, verbose=False, extra=(), check=False):
    """Builds libhdmc.so (check=True: the -DHDMC_CHECK debug build into
    _build_check/) and returns its path."""
    out_dir, lib = (CHECK_DIR, CHECK_LIB) if check else (OUT_DIR, LIB)
    if check:
        extra = tuple(extra) + ("-DHDMC_CHECK",)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    exe = nvcc()

    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [exe] + ARCH + FLAGS + list(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, r

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    for src, _, r in results:
        if verbose or r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on " + src)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + [o for _, o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link of libhdmc.so failed")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
