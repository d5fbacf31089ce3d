"""Build ``libxy.so`` (the C-ABI library) in-tree for sm_103a with nvcc.

Each ``csrc/*.cu`` translation unit is compiled in parallel, then linked into
one shared library next to this file.  No torch types cross the boundary.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libxy.so")
# The debug build: device-side index checks that record and skip (xy_debug.h).
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libxy_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force=False, verbose=False, extra=(), debug=False):
    """Build libxy.so (or, with debug=True, libxy_debug.so with -DXY_DEBUG)."""
    lib = LIB_DEBUG if debug else LIB
    bdir = BUILD_DEBUG if debug else BUILD
    if debug:
        extra = ("-DXY_DEBUG",) + tuple(extra)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    objs = []
    cmds = []
    for src in _sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmds.append([nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, len(cmds))) as ex:
        outs = list(ex.map(run, cmds))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    tmp = lib + ".tmp"
    run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, lib)
    return lib



def source_hash(files=("xy_fused.cu", "xy_device.cuh", "xy_tma.cuh")):
    """Hash of a kernel's own source files under csrc/ (ties an ncu capture to
    the kernel version it measured; the default is the fused sweep kernel)."""
    import hashlib
    h = hashlib.sha256()
    for name in files:
        p = os.path.join(CSRC, name)
        h.update(name.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(extra), extra=extra))

