"""Algorithmic work per launch, for the roofline of the leaf kernels.

Per-unit figures (method arithmetic, not the instructions a kernel happens to issue):
  residual pair (Laplace, potential and gradient): 22 + d_q operations, where d_q is the
      degree of the polynomial in r^2 that represents the residual function (the distance,
      r^2, the reciprocal square root, the polynomial, the potential and force updates);
  Chebyshev evaluation of the leaf expansion with its gradient: 2 p^3 FMA = 4 p^3 FLOP
      per target (sum-factorised contraction of the p^3 coefficients).
One launch of the residual kernel (k_pair) processes every visited pair once -- every
(target, source) pair of the direct lists -- and one launch of the expansion kernel
(k_leafexp) every target once.  The denominators are the pipe throughputs measured on the GPU
(paper_2606_27134_b300.peaks); the derived FP32 figure below is for comparison.
"""

# DRAM bytes (read + write) of one k_pair<float, Laplace, grad> launch at the benchmark
# workload from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel as
# it stands; None while the kernel has changed since its last capture.
PAIR_TRAFFIC_BYTES = 4.160e6

SMS = 148
FP32_LANES_PER_SM = 128
MAX_SM_GHZ = 2.032


def fp32_peak_tflops():
    """FP32 FMA pipe from unit counts: SMs x lanes x 2 FLOP x maximum SM clock."""
    return SMS * FP32_LANES_PER_SM * 2 * MAX_SM_GHZ / 1e3


def pair_flops(kernel, stats, grad=True):
    """Residual kernel: visited pairs x (22 + d_q) for Laplace with the gradient."""
    if kernel != "laplace":
        raise NotImplementedError("per-pair figure stated for the Laplace kernel")
    d_q = max(int(stats.get("fit_terms", 1)) - 1, 0)
    per_pair = (12 + d_q) + (10 if grad else 0)
    return float(stats["n_pairs"]) * per_pair


def leafexp_flops(stats, n_targets, grad=True):
    """Expansion kernel: targets x 4 p^3 (value and gradient)."""
    p = int(stats["p"])
    return float(n_targets) * (4 if grad else 2) * p ** 3
