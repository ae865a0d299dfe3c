"""Thin Python binding of libdmk_b300.so (the C ABI declared in include/dmk.h).

Argument marshalling only: every step of the evaluation runs in the CUDA library.  There is
no fallback: if the shared library is missing or cannot be loaded, every entry point raises.
PyTorch provides device memory and streams.
"""
import ctypes
import os

import numpy as np

from .build import LIB

KERNELS = {"laplace": 0, "stokeslet": 1, "stresslet": 2, "rotlet": 3}
D_RHO = {"laplace": 1, "stokeslet": 3, "stresslet": 9, "rotlet": 3}
D_U = {"laplace": 1, "stokeslet": 3, "stresslet": 3, "rotlet": 3}
PRECISIONS = {"fp64": 0, "mixed": 1}
STATUS = {0: "DMK_OK", 1: "DMK_ERR_INVALID_ARG", 2: "DMK_ERR_OUT_OF_DOMAIN", 3: "DMK_ERR_NOT_NEUTRAL",
          4: "DMK_ERR_UNSUPPORTED", 5: "DMK_ERR_TREE_DEPTH", 6: "DMK_ERR_OOM", 7: "DMK_ERR_CUDA",
          8: "DMK_ERR_TIMEOUT"}


# dmk_chi_reduce_fn: int (*)(double* chi, int64_t n, void* ctx)
CHI_REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_void_p)


class DmkError(RuntimeError):
    def __init__(self, status, detail):
        super().__init__(f"{STATUS.get(status, status)}: {detail}")
        self.status = status


class Stats(ctypes.Structure):
    _fields_ = [("c_times_1000", ctypes.c_int32), ("p", ctypes.c_int32), ("n_f", ctypes.c_int32),
                ("n_root_modes", ctypes.c_int32), ("n_levels", ctypes.c_int32), ("n_boxes", ctypes.c_int32),
                ("n_leaves", ctypes.c_int32), ("n_nonleaf", ctypes.c_int32), ("n_pairs", ctypes.c_int64),
                ("n_direct_entries", ctypes.c_int64), ("kernel_launches", ctypes.c_int32),
                ("fit_terms", ctypes.c_int32), ("stage_ms", ctypes.c_float * 10),
                ("n_capped_leaves", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_device_allocs", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("stage_ms", "reserved")}
        d["stage_ms"] = list(self.stage_ms)[:9]
        return d


class PlanInfo(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("s", ctypes.c_double), ("R", ctypes.c_double), ("dk", ctypes.c_double),
                ("p", ctypes.c_int32), ("n_f", ctypes.c_int32), ("n_root_modes", ctypes.c_int32),
                ("fit_terms_fp64", ctypes.c_int32), ("fit_terms_fp32", ctypes.c_int32),
                ("M", ctypes.c_int32 * 3), ("n_axis", ctypes.c_int32 * 3),
                ("d_rho", ctypes.c_int32), ("d_u", ctypes.c_int32), ("root_dft_len", ctypes.c_int32 * 6)]


_lib = None


def load(path=None):
    """Load the shared library (raises OSError if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise OSError(f"CUDA library not built: {path} (run paper_2606_27134_b300/build.py)")
    lib = ctypes.CDLL(path)
    vp, c_int, c_double, c_i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    dp = ctypes.POINTER(c_double)
    lib.dmk_plan.argtypes = [c_int, c_int, c_double, c_double, c_double, c_double, ctypes.POINTER(vp)]
    lib.dmk_plan_ex.argtypes = [c_int, c_int, dp, c_double, c_int, c_int, vp, ctypes.POINTER(vp)]
    lib.dmk_eval.argtypes = [vp, c_i64, vp, vp, vp, vp]
    lib.dmk_eval_host.argtypes = [vp, c_i64, vp, vp, vp, vp]
    lib.dmk_eval_static.argtypes = [vp, c_i64, vp, vp, vp, vp]
    lib.dmk_vjp.argtypes = [vp, c_i64, vp, vp, vp, vp, vp, vp]
    lib.dmk_eval_shard.argtypes = [vp, c_i64, c_i64, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int), CHI_REDUCE_FN,
                                   vp]
    lib.dmk_eval_targets.argtypes = [vp, c_i64, vp, vp, c_i64, vp, vp, vp]
    lib.dmk_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.dmk_set_timing.argtypes = [vp, c_int]
    lib.dmk_set_pair_overlap.argtypes = [vp, c_int, c_int]
    lib.dmk_destroy.argtypes = [vp]
    lib.dmk_plan_info.argtypes = [c_int, c_int, dp, c_double, ctypes.POINTER(PlanInfo)]
    lib.dmk_plan_table.argtypes = [c_int, c_int, dp, c_double, c_int, dp, c_i64, ctypes.POINTER(c_i64)]
    lib.dmk_status_string.argtypes = [c_int]
    lib.dmk_status_string.restype = ctypes.c_char_p
    lib.dmk_last_error.argtypes = [vp]
    lib.dmk_last_error.restype = ctypes.c_char_p
    for f in ("dmk_plan", "dmk_plan_ex", "dmk_eval", "dmk_eval_host", "dmk_eval_static", "dmk_vjp", "dmk_eval_shard",
              "dmk_eval_targets", "dmk_get_stats", "dmk_set_pair_overlap",
              "dmk_set_timing",
              "dmk_destroy", "dmk_plan_info", "dmk_plan_table"):
        getattr(lib, f).restype = c_int
    _lib = lib
    return lib


def _check(status, plan_ptr=None):
    if status != 0:
        lib = load()
        detail = lib.dmk_last_error(plan_ptr).decode()
        raise DmkError(status, detail)


class Plan:
    """dmk_plan_ex wrapper.  kernel in KERNELS, D in 0..3, L = (L1, L2, L3), tol in [1e-12, 1e-3]."""

    def __init__(self, kernel, D, L, tol, precision="mixed", n_s=250, stream=None):
        lib = load()
        self.kernel = kernel
        self.d_rho = D_RHO[kernel]
        self.d_u = D_U[kernel]
        Ls = (ctypes.c_double * 3)(*[float(v) for v in L])
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream is not None else None
        _check(lib.dmk_plan_ex(KERNELS[kernel], int(D), Ls, float(tol), PRECISIONS[precision], int(n_s), st,
                               ctypes.byref(h)), None)
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dmk_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_pair_overlap(self, enable=True, max_blocks_per_sm=0):
        """dmk_set_pair_overlap: the residual sums beside the far field (default) or in order."""
        _check(load().dmk_set_pair_overlap(self._h, 1 if enable else 0, int(max_blocks_per_sm)), self._h)

    def set_timing(self, on=True):
        _check(load().dmk_set_timing(self._h, 1 if on else 0), self._h)

    def stats(self):
        s = Stats()
        _check(load().dmk_get_stats(self._h, ctypes.byref(s)), self._h)
        return s.as_dict()

    def eval_ptr(self, N, points, strengths, potentials, grad=0):
        """Device pointers (ints) to N x 3, N x d_rho, N x d_u and optionally N x 3 x d_u FP64 arrays."""
        _check(load().dmk_eval(self._h, int(N), ctypes.c_void_p(points), ctypes.c_void_p(strengths),
                               ctypes.c_void_p(potentials), ctypes.c_void_p(grad) if grad else None), self._h)

    def eval(self, points, strengths, grad=False):
        """points (N,3), strengths (N, d_rho): CUDA FP64 torch tensors.  Returns (u, grad or None)."""
        import torch
        N = points.shape[0]
        pts = points.contiguous()
        rho = strengths.reshape(N, self.d_rho).contiguous()
        for t in (pts, rho):
            if not (t.is_cuda and t.dtype == torch.float64):
                raise TypeError("points and strengths must be CUDA float64 tensors")
        u = torch.empty((N, self.d_u), dtype=torch.float64, device=pts.device)
        g = torch.empty((N, 3, self.d_u), dtype=torch.float64, device=pts.device) if grad else None
        self.eval_ptr(N, pts.data_ptr(), rho.data_ptr(), u.data_ptr(), g.data_ptr() if grad else 0)
        return u, g

    def eval_targets(self, sources, strengths, targets, grad=False):
        """dmk_eval_targets: the sum over the sources (N,3) with strengths (N, d_rho) at separate
        targets (M,3); CUDA FP64 torch tensors.  Returns (u (M, d_u), grad (M, 3, d_u) or None)."""
        import torch
        N = sources.shape[0]
        M = targets.shape[0]
        src = sources.contiguous()
        rho = strengths.reshape(N, self.d_rho).contiguous()
        trg = targets.contiguous()
        for t in (src, rho, trg):
            if not (t.is_cuda and t.dtype == torch.float64):
                raise TypeError("sources, strengths and targets must be CUDA float64 tensors")
        u = torch.empty((M, self.d_u), dtype=torch.float64, device=trg.device)
        g = torch.empty((M, 3, self.d_u), dtype=torch.float64, device=trg.device) if grad else None
        vp = ctypes.c_void_p
        _check(load().dmk_eval_targets(self._h, N, vp(src.data_ptr()), vp(rho.data_ptr()), M, vp(trg.data_ptr()),
                                       vp(u.data_ptr()), vp(g.data_ptr()) if grad else None), self._h)
        return u, g

    def vjp(self, points, strengths, grad_u, g, want_strengths=True, want_points=True):
        """dmk_vjp: (dL/dstrengths (N, d_rho) or None, dL/dpoints (N, 3) or None) for the upstream
        gradient g = dL/du (N, d_u); grad_u is the field gradient returned by the forward eval.
        CUDA float64 tensors."""
        import torch
        N = points.shape[0]
        pts = points.contiguous()
        rho = strengths.reshape(N, self.d_rho).contiguous()
        gg = g.reshape(N, self.d_u).contiguous()
        for t in (pts, rho, gg):
            if not (t.is_cuda and t.dtype == torch.float64):
                raise TypeError("points, strengths and g must be CUDA float64 tensors")
        gu = grad_u.contiguous() if want_points else None
        if want_points and not (gu.is_cuda and gu.dtype == torch.float64 and gu.numel() == N * 3 * self.d_u):
            raise TypeError("grad_u must be the (N, 3, d_u) CUDA float64 field gradient of the forward eval")
        ds = torch.empty((N, self.d_rho), dtype=torch.float64, device=pts.device) if want_strengths else None
        dx = torch.empty((N, 3), dtype=torch.float64, device=pts.device) if want_points else None
        vp = ctypes.c_void_p
        _check(load().dmk_vjp(self._h, N, vp(pts.data_ptr()), vp(rho.data_ptr()),
                              vp(gu.data_ptr()) if want_points else None, vp(gg.data_ptr()),
                              vp(ds.data_ptr()) if want_strengths else None,
                              vp(dx.data_ptr()) if want_points else None), self._h)
        return ds, dx

    def eval_host(self, points, strengths, grad=False):
        """Host numpy arrays in, host numpy arrays out (copies inside the library)."""
        pts = np.ascontiguousarray(points, dtype=np.float64)
        N = pts.shape[0]
        rho = np.ascontiguousarray(np.asarray(strengths, dtype=np.float64).reshape(N, self.d_rho))
        u = np.empty((N, self.d_u))
        g = np.empty((N, 3, self.d_u)) if grad else None
        _check(load().dmk_eval_host(self._h, N, pts.ctypes.data, rho.ctypes.data, u.ctypes.data,
                                    g.ctypes.data if grad else None), self._h)
        return u, g

    def eval_host_ptr(self, N, points, strengths, potentials, grad=0):
        """Host pointers (ints, e.g. of pinned torch tensors)."""
        _check(load().dmk_eval_host(self._h, int(N), ctypes.c_void_p(points), ctypes.c_void_p(strengths),
                                    ctypes.c_void_p(potentials), ctypes.c_void_p(grad) if grad else None), self._h)


def plan_info(kernel, D, L, tol):
    """Host-only plan parameters (dmk_plan_info)."""
    lib = load()
    out = PlanInfo()
    Ls = (ctypes.c_double * 3)(*[float(v) for v in L])
    _check(lib.dmk_plan_info(KERNELS[kernel], int(D), Ls, float(tol), ctypes.byref(out)), None)
    d = {k: getattr(out, k) for k, _ in out._fields_}
    d["M"] = list(out.M)
    d["n_axis"] = list(out.n_axis)
    d["root_dft_len"] = [list(out.root_dft_len)[:3], list(out.root_dft_len)[3:]]
    return d


def plan_table(kernel, D, L, tol, which):
    """Host-only plan table (dmk_plan_table) as a numpy array."""
    lib = load()
    Ls = (ctypes.c_double * 3)(*[float(v) for v in L])
    n = ctypes.c_int64()
    _check(lib.dmk_plan_table(KERNELS[kernel], int(D), Ls, float(tol), int(which), None, 0, ctypes.byref(n)), None)
    buf = np.empty(n.value)
    _check(lib.dmk_plan_table(KERNELS[kernel], int(D), Ls, float(tol), int(which),
                              buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value, ctypes.byref(n)), None)
    return buf


def status_string(code):
    return load().dmk_status_string(int(code)).decode()


def last_plan_error():
    return load().dmk_last_error(None).decode()
