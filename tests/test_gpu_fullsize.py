"""The full workload sizes.

The benchmark workload itself (Laplace 2P slab, N = 1e5, n_s = 250, the inputs bench.py
times, on a side stream like bench.py) is compared with the oracle element by element at
2000 sampled targets (tests/golden/fullsize_laplace_2P_N1e5.npz, written by
tests/golden/make_fullsize_samples.py from the oracle alone), with identical forests.

Where the oracle cannot run the whole evaluation (N = 1e6 and 4e6), element-by-element
parity is established at smaller sizes (test_gpu_parity.py) and these tests check what holds
at any size:
  * the mixed path agrees with the plain FP64 path within the mixed-path bar (1e-5);
  * linearity in the strengths (to roundoff, same tree);
  * invariance under a translation by a vector in the periodic directions (the forest
    changes, so agreement is to the tolerance row);
  * finite, well-formed outputs and the expected forest statistics.
Configurations follow the benchmark workloads (uniform slab for Laplace 2P N=1e5, Stokeslet
1P aspect 8 N=1e6, adaptive clustered Laplace 3P N=1e6, stresslet and rotlet 3P on 16 cubes
stacked along x3 with N=4e6).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_27134_b300 import dmk, workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(torch.linalg.norm((a - b).ravel()) / torch.linalg.norm(b.ravel()))


def run(kernel, D, L, tol, x, rho, prec, n_s=250):
    plan = dmk.Plan(kernel, D, L, tol, precision=prec, n_s=n_s)
    u, g = plan.eval(x, rho, grad=True)
    torch.cuda.synchronize()
    st = plan.stats()
    plan.close()
    return u, g, st


CONFIGS = [
    ("laplace-2P-slab-1e5", "laplace", 2, [1.0, 1.0, 0.25], 1e-6, 100_000, "uniform"),
    ("stokeslet-1P-aspect8-1e6", "stokeslet", 1, [8.0, 1.0, 1.0], 1e-6, 1_000_000, "uniform"),
    ("laplace-3P-clustered-1e6", "laplace", 3, [1.0, 1.0, 1.0], 1e-6, 1_000_000, "clusters"),
    ("stresslet-3P-16cubes-4e6", "stresslet", 3, [1.0, 1.0, 16.0], 1e-6, 4_000_000, "uniform"),
    ("rotlet-3P-16cubes-4e6", "rotlet", 3, [1.0, 1.0, 16.0], 1e-6, 4_000_000, "uniform"),
]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_laplace_2P_N1e5.npz")


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_benchmark_workload_matches_oracle_samples(prec, bar):
    ref = np.load(GOLDEN)
    N, L = 100_000, [1.0, 1.0, 0.25]
    dev = torch.device("cuda", 0)
    assert list(ref["seeds"][:2]) == [2002, 3002]
    xt = torch.tensor(W.uniform_points(N, L, 2002), dtype=torch.float64, device=dev)
    qt = torch.tensor(W.uniform_charges(N, 3002), dtype=torch.float64, device=dev).reshape(N, 1)
    stream = torch.cuda.Stream(device=dev)
    plan = dmk.Plan("laplace", 2, L, 1e-6, precision=prec, n_s=250, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        u, g = plan.eval(xt, qt, grad=True)
    torch.cuda.synchronize()
    st = plan.stats()
    plan.close()
    assert (st["n_boxes"], st["n_leaves"], st["n_levels"]) == (int(ref["n_boxes"]), int(ref["n_leaves"]),
                                                                 int(ref["n_levels"]))
    idx = torch.tensor(ref["idx"], device=dev)
    us, gs = u[idx].cpu().numpy(), g[idx].cpu().numpy()
    eu = np.linalg.norm(us - ref["u"]) / np.linalg.norm(ref["u"])
    eg = np.linalg.norm(gs - ref["grad"]) / np.linalg.norm(ref["grad"])
    assert eu <= bar and eg <= bar, (eu, eg)


@pytest.mark.parametrize("cfg", CONFIGS, ids=[c[0] for c in CONFIGS])
def test_fullsize_properties(cfg):
    cid, kernel, D, L, tol, N, gen = cfg
    dev = torch.device("cuda", 0)
    if gen == "uniform":
        x = W.uniform_points(N, L, 4001)
    else:
        x = W.clustered_points(N, L, 4001, n_centers=64, sigma=0.02)
    if kernel == "laplace":
        rho = (W.uniform_charges(N, 4002) if D < 3 else W.balanced_charges(N, 4002)).reshape(N, 1)
    else:
        rho = W.stokes_strengths(kernel, N, 4002)
    xt = torch.tensor(x, dtype=torch.float64, device=dev)
    rt = torch.tensor(rho, dtype=torch.float64, device=dev)
    del x, rho
    u64, g64, st = run(kernel, D, L, tol, xt, rt, "fp64")
    assert torch.isfinite(u64).all() and torch.isfinite(g64).all()
    u32, g32, st32 = run(kernel, D, L, tol, xt, rt, "mixed")
    assert st32["n_boxes"] == st["n_boxes"]
    assert rel(u32, u64) <= 1e-5 and rel(g32, g64) <= 1e-5
    del u32, g32
    torch.cuda.empty_cache()
    # linearity (same tree): u(-2 rho) = -2 u(rho)
    u2, g2, _ = run(kernel, D, L, tol, xt, -2 * rt, "fp64")
    assert rel(u2, -2 * u64) <= 1e-13
    # translation by a vector in the periodic directions
    shift = torch.tensor([0.3711 * L[0] if D > 0 else 0.0, 0.6173 * L[1] if D > 1 else 0.0,
                          0.2293 * L[2] if D > 2 else 0.0], dtype=torch.float64, device=dev)
    ut, gt, _ = run(kernel, D, L, tol, xt + shift, rt, "fp64")
    assert rel(ut, u64) <= 10 * tol and rel(gt, g64) <= 10 * tol
