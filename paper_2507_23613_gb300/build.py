"""Build libmfwh.so in-tree for sm_103a with nvcc (and g++ for host-only sources).

Translation units compile in parallel into ``_build/``; the shared library is
linked next to this file.  A rebuild happens when any source or header is newer
than the library.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmfwh.so")
# the index-checked debugging build (-DMFWH_BOUNDS_CHECK, csrc/check.cuh)
BUILD_BC = os.path.join(HERE, "_build_bc")
LIB_BC = os.path.join(HERE, "libmfwh_bc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmfwh")


def _sources():
    srcs = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return [os.path.join(CSRC, s) for s in srcs], hdrs


def needs_build(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    srcs, hdrs = _sources()
    return any(os.path.getmtime(p) > t for p in srcs + hdrs + [os.path.abspath(__file__)])


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force=False, verbose=False, bounds_check=False):
    """Compile every CUDA/C++ source of libmfwh for sm_103a; returns the library path.
    bounds_check: the index-checked debugging build libmfwh_bc.so (-DMFWH_BOUNDS_CHECK)."""
    lib, bdir = (LIB_BC, BUILD_BC) if bounds_check else (LIB, BUILD)
    if not force and not needs_build(lib):
        return lib
    nvcc = _nvcc()
    os.makedirs(bdir, exist_ok=True)
    srcs, _ = _sources()
    extra = ["-DMFWH_BOUNDS_CHECK"] if bounds_check else []
    jobs = []
    for s in srcs:
        obj = os.path.join(bdir, os.path.basename(s) + ".o")
        if s.endswith(".cu"):
            cmd = [nvcc, "-c", s, "-o", obj] + NVCC_FLAGS + extra
        else:
            cmd = [os.environ.get("CXX", "g++"), "-c", s, "-o", obj] + CXX_FLAGS + extra
        jobs.append((cmd, obj))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o, file=sys.stderr)
    tmp = lib + ".tmp"
    _run([nvcc, "-shared", "-o", tmp] + [o for _, o in jobs] + ARCH + ["-lcudart_static", "-lpthread", "-ldl"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
