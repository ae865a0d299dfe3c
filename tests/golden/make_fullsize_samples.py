"""Writes tests/golden/fullsize_laplace_2P_N1e5.npz: oracle values at sampled targets of the
full-size benchmark workload (Laplace, D = 2, L = (1, 1, 0.25), N = 1e5 uniform points, neutral
uniform charges, tol 1e-6, n_s = 250; the inputs are those bench.py times, seeds 2002/3002).

Calls only oracle/ and the seeded input generators (no CUDA code).  The oracle evaluates the
whole problem (forest, upward pass, root far field, plane waves) and runs its leaf step for
the sampled targets only (oracle.dmk.evaluate(targets=...)), so each stored value is the one
the full evaluation gives.  Also stored: the forest's box, leaf and level counts.

    python tests/golden/make_fullsize_samples.py        (about a minute on one core)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.dmk import evaluate                       # noqa: E402
from paper_2606_27134_b300 import workloads as W      # noqa: E402

N, L, D, TOL, NS = 100_000, [1.0, 1.0, 0.25], 2, 1e-6, 250
N_SAMPLE, SAMPLE_SEED = 2000, 2024


def main():
    x = W.uniform_points(N, L, 2002)
    q = W.uniform_charges(N, 3002)
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(N, N_SAMPLE, replace=False))
    t = time.time()
    r = evaluate("laplace", D, L, TOL, x, q, n_s=NS, grad=True, targets=idx)
    f = r.forest
    out = os.path.join(HERE, "fullsize_laplace_2P_N1e5.npz")
    np.savez_compressed(out, idx=idx, u=r.u[idx], grad=r.grad[idx],
                        n_boxes=len(f.by_id), n_leaves=len(f.leaves()), n_levels=f.nlevels,
                        seeds=np.array([2002, 3002, SAMPLE_SEED]))
    print(out, "%.1f s" % (time.time() - t), len(f.by_id), len(f.leaves()), f.nlevels)


if __name__ == "__main__":
    main()
