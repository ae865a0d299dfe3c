"""Measured arithmetic peaks of the GPU (libdmk_peaks.so), the denominators of the ALU
roofline fractions.

Three pipes bound the DMK kernels: the FP32 FMA pipe (residual sums and the Chebyshev and
plane-wave contractions of the mixed path), the FP64 FMA pipe (the plain path and the root
far field) and the MUFU reciprocal square root (one per residual pair).  Each is timed with
CUDA events, best of a few launches of about 20 ms, with the SM clock sampled by nvidia-smi
while the launches run.  The GPU's clocks and settings are only read, never changed.

Derived figures for comparison (unit counts x maximum SM clock, 148 SMs at 2.032 GHz):
FP32 FMA 128 lanes/SM -> 77.0 TFLOP/s; MUFU 16/SM/clock -> 4.81 Tops/s.
"""
import ctypes
import os
import statistics
import subprocess
import tempfile
import time

from .build import PEAKS_LIB

_PIPES = {"fp32_ffma": (0, 20000), "fp64_dfma": (1, 300), "mufu_rsqrt": (2, 2500)}


def _load():
    if not os.path.exists(PEAKS_LIB):
        raise OSError(f"peaks library not built: {PEAKS_LIB}")
    lib = ctypes.CDLL(PEAKS_LIB)
    lib.dmk_peak_measure.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.dmk_peak_measure.restype = ctypes.c_int
    return lib


def _one(lib, which, iters, reps):
    ops, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib.dmk_peak_measure(which, iters, reps, ctypes.byref(ops), ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError(f"dmk_peak_measure({which}) failed with CUDA error {rc}")
    return ops.value, ms.value


def _sample_clocks(index, path):
    q = "clocks.sm,clocks.max.sm,clocks_event_reasons.active"
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                              "-lms", "50"], stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def measure(device_index=0, target_ms=20.0, reps=5):
    """{"fp32_tflops", "fp64_tflops", "mufu_rsqrt_tops", "ms": {...}, "clocks": {...}} on the current device."""
    lib = _load()
    out, times = {}, {}
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "clk.csv")
        proc, fh = _sample_clocks(device_index, path)
        time.sleep(0.2)
        for name, (which, iters) in _PIPES.items():
            # size the launch to about target_ms from one probe launch
            _, ms = _one(lib, which, max(1, iters // 10), 1)
            iters2 = max(1, int(iters // 10 * target_ms / max(ms, 1e-3)))
            ops, ms = _one(lib, which, iters2, reps)
            out[name] = ops
            times[name] = ms
        if proc:
            proc.terminate()
            try:
                proc.wait(timeout=5)
            except Exception:
                proc.kill()
            fh.close()
        sm, mx = [], None
        try:
            for line in open(path):
                f = [v.strip() for v in line.split(",")]
                try:
                    sm.append(float(f[0]))
                    mx = float(f[1])
                except (ValueError, IndexError):
                    pass
        except FileNotFoundError:
            pass
    return {"fp32_tflops": out["fp32_ffma"] / 1e12, "fp64_tflops": out["fp64_dfma"] / 1e12,
            "mufu_rsqrt_tops": out["mufu_rsqrt"] / 1e12, "ms": times,
            "clocks": {"sm_mhz_median": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                       "samples": len(sm)},
            "how": "dmk_peak_measure: 4 x 512-thread blocks per SM, 8 independent FMA/rsqrt chains per thread, "
                   "best of %d CUDA-event-timed launches of ~%g ms" % (reps, target_ms)}


if __name__ == "__main__":
    import json
    import torch

    torch.cuda.init()
    print(json.dumps(measure()))
