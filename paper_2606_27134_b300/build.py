"""Builds libdmk_b300.so (the DMK library) and libdmk_peaks.so (pipe-throughput
microbenchmarks used for the roofline denominators) in this package directory with nvcc for
sm_103a."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libdmk_b300.so")
PEAKS_LIB = os.path.join(HERE, "libdmk_peaks.so")
PEAKS_SOURCES = ["dmk_peaks.cu"]
SOURCES = ["dmk_plan.cpp", "dmk_api.cu"]
HEADERS = ["dmk_internal.h", "dmk_device.cuh", "dmk_tree.cuh", "dmk_kernels.cuh", "dmk_fast.cuh"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def up_to_date(lib=LIB, sources=None, headers=None):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in (SOURCES + HEADERS if sources is None else sources + (headers or []))]
    deps.append(os.path.join(HERE, "..", "include", "dmk.h"))
    return all(os.path.getmtime(d) <= t for d in deps if os.path.exists(d))


def _nvcc_shared(lib, sources, verbose, extra):
    cmd = [nvcc(), "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-lineinfo",
           "-gencode", "arch=compute_103a,code=sm_103a", "--expt-relaxed-constexpr",
           "-I", os.path.join(HERE, "..", "include"), *extra,
           "-o", lib + ".tmp"] + [os.path.join(CSRC, f) for f in sources]
    if verbose:
        print(" ".join(cmd))
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


def build_peaks(force=False, verbose=False, extra=()):
    if force or not up_to_date(PEAKS_LIB, PEAKS_SOURCES, []):
        _nvcc_shared(PEAKS_LIB, PEAKS_SOURCES, verbose, extra)
    return PEAKS_LIB


def build(force=False, verbose=False, extra=()):
    build_peaks(force, verbose, extra)
    if not force and up_to_date():
        return LIB
    return _nvcc_shared(LIB, SOURCES, verbose, extra)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=[a for a in sys.argv[1:] if a != "--force"])
    print(LIB)
