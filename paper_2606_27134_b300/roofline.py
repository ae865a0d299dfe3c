"""Algorithmic work per launch and the FP32 ALU peak used for the leaf-kernel roofline.

Per-unit figures (method arithmetic, not the instructions a kernel happens to issue):
  residual pair (Laplace, potential and gradient): 22 + d_q operations, where d_q is the
      degree of the polynomial in r^2 that represents the residual function (the distance,
      r^2, the reciprocal square root, the polynomial, the potential and force updates);
  Chebyshev evaluation of the leaf expansion with its gradient: 2 p^3 FMA = 4 p^3 FLOP
      per target (sum-factorised contraction of the p^3 coefficients).
One leaf-kernel launch processes every visited pair and every target once.
"""

# DRAM bytes (read + write) of one k_leaf3<float, Laplace, grad> launch at the benchmark
# workload, from one ncu capture of the kernel as it stands (profiles/k_leaf3_laplace_2P_N1e5_mixed.md);
# set to None whenever the kernel changes until it is captured again.
LEAF_TRAFFIC_BYTES = 37.22e6 + 0.017e6

SMS = 148
FP32_LANES_PER_SM = 128
MAX_SM_GHZ = 2.032


def fp32_peak_tflops():
    """FP32 FMA pipe: SMs x lanes x 2 FLOP x maximum SM clock."""
    return SMS * FP32_LANES_PER_SM * 2 * MAX_SM_GHZ / 1e3


def leaf_flops(kernel, stats, n_targets, grad=True, precision="mixed"):
    if kernel != "laplace":
        raise NotImplementedError("per-pair figure stated for the Laplace kernel")
    d_q = max(int(stats.get("fit_terms", 1)) - 1, 0)
    per_pair = (12 + d_q) + (10 if grad else 0)
    p = int(stats["p"])
    per_target = (4 if grad else 2) * p ** 3
    return float(stats["n_pairs"]) * per_pair + float(n_targets) * per_target
