"""Build the in-tree CUDA library (sm_103a) with nvcc.

    python -m paper_1812_03358_b300.build

produces paper_1812_03358_b300/_lib/liblt.so from csrc/*.cu and csrc/*.cpp,
and beside it the test build _lib/liblt_testhooks.so (the same sources with
-DLT_TEST_HOOKS: it adds the fault-injection entry points of
include/lt_testing.h, which the product library does not carry).  The two
are compiled concurrently.
"""
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "liblt.so")
TEST_LIB = os.path.join(LIBDIR, "liblt_testhooks.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(ROOT, "include", "*.h")))


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in sources() + headers() + [__file__])


def _command(out, verbose, extra):
    return [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
            "-Xcompiler", "-fvisibility=hidden", "-Xptxas", "-v" if verbose else "-O3",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra,
            *sources(), "-o", out, "-lcudart"]


def build(force=False, verbose=False, extra=()):
    """Builds whichever of liblt.so and liblt_testhooks.so is out of date;
    returns the product library's path."""
    os.makedirs(LIBDIR, exist_ok=True)
    jobs = []
    for lib, flags in ((LIB, ()), (TEST_LIB, ("-DLT_TEST_HOOKS",))):
        if force or not up_to_date(lib):
            tmp = lib + ".tmp"
            jobs.append((lib, tmp, subprocess.Popen(_command(tmp, verbose, (*flags, *extra)),
                                                    stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    failed = None
    for lib, tmp, proc in jobs:
        out, err = proc.communicate()
        if proc.returncode != 0:
            failed = failed or (lib, out + err)
            continue
        if verbose:
            sys.stderr.write(err)
        os.replace(tmp, lib)
    if failed:
        sys.stderr.write(failed[1])
        raise RuntimeError(f"nvcc failed building {os.path.basename(failed[0])}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
