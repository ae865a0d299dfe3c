"""dmk_eval_targets (targets apart from the sources) against the oracle's evaluate_targets,
element by element: relative l2 <= 1e-10 on the plain FP64 path, <= 1e-5 on the mixed path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dmk import evaluate_targets
from paper_2606_27134_b300 import dmk, workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ("laplace-2P-slab", "laplace", 2, [1, 1, 0.25], 2500, 900, 40),
    ("laplace-3P-nonexact", "laplace", 3, [1, 1.3, 1.7], 2000, 700, 40),
    ("stokeslet-1P", "stokeslet", 1, [4, 1, 1], 1500, 600, 30),
    ("rotlet-3P-four-cubes", "rotlet", 3, [1, 1, 4], 1500, 600, 30),
    ("stresslet-2P", "stresslet", 2, [1, 1, 1], 800, 400, 30),
]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def inputs(kernel, D, L, N, M, seed):
    x = W.mixed_points(N, L, seed, D=D)
    q = W.stokes_strengths(kernel, N, seed + 1)
    y = W.uniform_points(M, L, seed + 2)
    return x, q, y


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("mixed", 1e-5)])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_targets_match_oracle(case, precision, bar):
    _, kernel, D, L, N, M, n_s = case
    x, q, y = inputs(kernel, D, L, N, M, 501)
    ref = evaluate_targets(kernel, D, L, 1e-6, x, q, y, n_s=n_s, grad=True)
    p = dmk.Plan(kernel, D, L, 1e-6, precision=precision, n_s=n_s)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    u, g = p.eval_targets(dev(x), dev(q), dev(y), grad=True)
    u, g = u.cpu().numpy(), g.cpu().numpy()
    assert u.shape == ref.u.shape
    assert rel(u, ref.u) < bar
    assert rel(g, ref.grad) < bar
    p.close()


def test_targets_without_sources_or_targets():
    p = dmk.Plan("laplace", 3, [1, 1, 1], 1e-6, n_s=40)
    y = torch.tensor(W.uniform_points(50, [1, 1, 1], 511), device="cuda")
    e = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    u, g = p.eval_targets(e, torch.zeros((0, 1), dtype=torch.float64, device="cuda"), y, grad=True)
    assert torch.count_nonzero(u) == 0 and torch.count_nonzero(g) == 0
    x = torch.tensor(W.uniform_points(100, [1, 1, 1], 512), device="cuda")
    q = torch.tensor(W.neutral_charges(100, 513), device="cuda")
    u, _ = p.eval_targets(x, q, e)
    assert u.shape == (0, 1)
    p.close()


def test_targets_out_of_domain_is_reported():
    p = dmk.Plan("laplace", 2, [1, 1, 0.5], 1e-6, n_s=40)
    x = torch.tensor(W.uniform_points(100, [1, 1, 0.5], 521), device="cuda")
    q = torch.tensor(W.neutral_charges(100, 522), device="cuda")
    y = torch.tensor([[0.5, 0.5, 0.75]], dtype=torch.float64, device="cuda")      # free x3 beyond L3
    with pytest.raises(dmk.DmkError) as e:
        p.eval_targets(x, q, y)
    assert e.value.status == 2
    p.close()
