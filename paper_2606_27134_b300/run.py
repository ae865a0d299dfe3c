"""Evaluate one synthetic workload through the library, for timing and profiling runs.

    python -m paper_2606_27134_b300.run --kernel stresslet --D 3 --L 1 1 16 --N 1000000 --reps 2

Points and strengths come from workloads.py (uniform points, the paper's "half uniform, half
clustered" mix, Gaussian clusters or the pipe; the kernel's strength distribution with seeds
7001/7002, the ones bench.py uses); the evaluation runs on cuda:0 with potentials and gradients
and prints the per-stage CUDA-event times of each repetition.
"""
import argparse
import time

import numpy as np


def make_inputs(kernel, D, L, N, points="uniform"):
    from . import workloads as W
    if points == "uniform":
        x = W.uniform_points(N, L, 7001)
    elif points == "mixed":
        x = W.mixed_points(N, L, 7001, D=D)
    elif points == "clusters":
        x = W.clustered_points(N, L, 7001, n_centers=64, sigma=0.02)
    elif points == "pipe":
        x = W.cylinder_points(L[0], per_unit=int(round(N / L[0])))
    else:
        raise ValueError(points)
    n = x.shape[0]
    if kernel == "laplace":
        rho = (W.uniform_charges(n, 7002) if D < 3 else W.balanced_charges(n, 7002)).reshape(n, 1)
    else:
        rho = W.stokes_strengths(kernel, n, 7002)
    return x, rho


def main(argv=None):
    import torch
    from . import dmk
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--kernel", default="laplace", choices=list(dmk.KERNELS))
    ap.add_argument("--D", type=int, default=2)
    ap.add_argument("--L", type=float, nargs=3, default=[1.0, 1.0, 0.25])
    ap.add_argument("--N", type=int, default=100000)
    ap.add_argument("--points", default="uniform", choices=["uniform", "mixed", "clusters", "pipe"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n_s", type=int, default=250)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--no-grad", action="store_true")
    a = ap.parse_args(argv)
    x, rho = make_inputs(a.kernel, a.D, a.L, a.N, a.points)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    rt = torch.tensor(rho, dtype=torch.float64, device="cuda")
    plan = dmk.Plan(a.kernel, a.D, a.L, a.tol, precision=a.precision, n_s=a.n_s)
    plan.set_timing(True)
    for i in range(a.reps):
        t = time.perf_counter()
        u, g = plan.eval(xt, rt, grad=not a.no_grad)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t) * 1e3
        st = plan.stats()
        stages = dict(zip(("tree", "upward", "root", "planewave", "shift", "leaf", "total", "leaf_pair",
                           "leaf_exp"), (round(v, 3) for v in st["stage_ms"])))
        print(f"rep {i}: N={x.shape[0]} wall {wall:.3f} ms, stages {stages}, boxes {st['n_boxes']}, "
              f"levels {st['n_levels']}, pairs {st['n_pairs']}", flush=True)
    plan.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
