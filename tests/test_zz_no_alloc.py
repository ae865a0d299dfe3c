"""dmk_eval_static: the evaluation without device allocation, for callers that cannot call
cudaMalloc while they evaluate (applications whose device memory is held by their own
memory pool).  It must return what dmk_eval returns, on consecutive calls that share its
static workspace, and reject problems beyond its stated limits.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_27134_b300 import dmk, workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    # kernel, D, L, precision, N, n_s, tolerance (the parity bars of the GPU tests)
    ("laplace", 3, [1, 1, 1], "mixed", 3000, 60, 1e-5),
    ("laplace", 2, [1, 1, 0.5], "fp64", 1200, 80, 1e-10),
    ("stokeslet", 1, [2, 1, 1], "mixed", 1500, 200, 1e-5),
]


def call(lib, fn, plan, N, x, rho, u, g):
    return getattr(lib, fn)(plan._h, N, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
                            ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(g.data_ptr()))


def rel(a, b):
    return float(torch.linalg.norm((a - b).ravel()) / torch.linalg.norm(b.ravel()))


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}P-{c[3]}" for c in CASES])
def test_static_matches_allocating_entry_point(case):
    kernel, D, L, prec, N, n_s, bar = case
    lib = dmk.load()
    # a fresh plan whose first evaluations go through dmk_eval_static: the plan's allocation
    # count (tables only) must not move, and a second plan gives the allocating reference
    plan = dmk.Plan(kernel, D, L, 1e-6, precision=prec, n_s=n_s)
    ref = dmk.Plan(kernel, D, L, 1e-6, precision=prec, n_s=n_s)
    dev = torch.device("cuda", 0)
    allocs = plan.stats()["n_device_allocs"]
    assert allocs > 0                     # the plan's tables
    inputs = []
    for seed in (11, 12):
        inputs.append((torch.tensor(W.mixed_points(N, L, seed, D=D), dtype=torch.float64, device=dev),
                       torch.tensor(W.stokes_strengths(kernel, N, seed + 1), dtype=torch.float64, device=dev)))
    out = []
    for x, rho in inputs:      # two calls in a row: the shared array keeps the previous contents
        u1 = torch.full((N, plan.d_u), float("nan"), dtype=torch.float64, device=dev)
        g1 = torch.full((N, 3, plan.d_u), float("nan"), dtype=torch.float64, device=dev)
        st = call(lib, "dmk_eval_static", plan, N, x, rho, u1, g1)
        assert st == 0, lib.dmk_last_error(plan._h).decode()
        torch.cuda.synchronize()
        assert plan.stats()["n_device_allocs"] == allocs
        out.append((u1, g1))
    for (x, rho), (u1, g1) in zip(inputs, out):
        u0 = torch.empty((N, plan.d_u), dtype=torch.float64, device=dev)
        g0 = torch.empty((N, 3, plan.d_u), dtype=torch.float64, device=dev)
        assert call(lib, "dmk_eval", ref, N, x, rho, u0, g0) == 0, lib.dmk_last_error(ref._h)
        torch.cuda.synchronize()
        assert torch.isfinite(u1).all() and torch.isfinite(g1).all()
        # the same kernels in the same order on the same inputs: identical results
        assert torch.equal(u1, u0) and torch.equal(g1, g0), (rel(u1, u0), rel(g1, g0), bar)
    assert not torch.equal(out[0][0], out[1][0])
    # after the allocating plan has run, the static entry point still matches it
    x, rho = inputs[0]
    u1 = torch.full((N, plan.d_u), float("nan"), dtype=torch.float64, device=dev)
    g1 = torch.full((N, 3, plan.d_u), float("nan"), dtype=torch.float64, device=dev)
    assert call(lib, "dmk_eval_static", ref, N, x, rho, u1, g1) == 0
    torch.cuda.synchronize()
    assert torch.equal(u1, out[0][0]) and torch.equal(g1, out[0][1])
    plan.close()
    ref.close()


def test_static_rejects_oversize_problems():
    lib = dmk.load()
    plan = dmk.Plan("laplace", 3, [1, 1, 1], 1e-6, precision="mixed")
    N = 16385
    dev = torch.device("cuda", 0)
    x = torch.rand((N, 3), dtype=torch.float64, device=dev)
    q = torch.zeros((N, 1), dtype=torch.float64, device=dev)
    u = torch.empty((N, 1), dtype=torch.float64, device=dev)
    g = torch.empty((N, 3, 1), dtype=torch.float64, device=dev)
    assert call(lib, "dmk_eval_static", plan, N, x, q, u, g) == 1
    assert b"16384" in lib.dmk_last_error(plan._h)
    # a problem whose workspace exceeds the static array: FP64 at tol 1e-12 (p = 38)
    big = dmk.Plan("laplace", 3, [1, 1, 1], 1e-12, precision="fp64", n_s=8)
    N = 16000
    x = torch.tensor(W.uniform_points(N, [1, 1, 1], 5), dtype=torch.float64, device=dev)
    q = torch.tensor(W.neutral_charges(N, 6), dtype=torch.float64, device=dev).reshape(N, 1)
    u = torch.empty((N, 1), dtype=torch.float64, device=dev)
    g = torch.empty((N, 3, 1), dtype=torch.float64, device=dev)
    assert call(lib, "dmk_eval_static", big, N, x, q, u, g) == 6
    assert b"static workspace" in lib.dmk_last_error(big._h)
    plan.close()
    big.close()
