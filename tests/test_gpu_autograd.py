"""Forces through torch.autograd (backward = one more evaluation of the hot path) checked
against the oracle's analytic gradient and against central finite differences of the energy."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dmk import evaluate
from oracle.tree import BITS
from paper_2606_27134_b300 import autograd as ag, workloads as W

pytestmark = pytest.mark.gpu


def test_forces_match_oracle_gradient():
    N, L, D = 1500, [1.0, 1.0, 1.0], 3
    x = W.clustered_points(N, L, seed=71, n_centers=8, sigma=0.03)
    q = W.balanced_charges(N, seed=72)
    ref = evaluate("laplace", D, L, 1e-6, x, q, n_s=30, grad=True)
    F_ref = -q[:, None] * ref.grad[:, :, 0]
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q, dtype=torch.float64, device="cuda")
    for prec, bar in (("fp64", 1e-10), ("mixed", 1e-5)):
        E, F = ag.energy_and_forces(xt, qt, D, L, 1e-6, precision=prec, n_s=30)
        F = F.cpu().numpy()
        assert np.linalg.norm(F - F_ref) / np.linalg.norm(F_ref) <= bar
        E_ref = 0.5 * np.sum(q * ref.u[:, 0])
        assert abs(float(E) - E_ref) <= bar * abs(E_ref) * 10


def test_strength_gradient_is_potential():
    N, L, D = 1200, [1.0, 1.0, 0.5], 2
    x = W.uniform_points(N, L, seed=81)
    q = W.uniform_charges(N, seed=82)
    pot = ag.Potential("laplace", D, L, 1e-6, precision="fp64", n_s=40)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q, dtype=torch.float64, device="cuda").reshape(N, 1).requires_grad_(True)
    u = pot(xt, qt)
    E = 0.5 * (qt * u).sum()
    (gq,) = torch.autograd.grad(E, qt)
    assert torch.allclose(gq, u.detach(), rtol=1e-9, atol=1e-12 * float(u.abs().max()))


def test_forces_finite_difference():
    """Central differences of the FP64 energy on points far from every grid line (fixed tree);
    agreement to 10x the tolerance row: the adjoint gives the gradient of the exact sum, the
    difference quotient that of its eps-approximation."""
    N, L, D, tol = 2000, [1.0, 1.0, 1.0], 3, 1e-6
    x = W.clustered_points(N, L, seed=91, n_centers=8, sigma=0.05)
    q = W.balanced_charges(N, seed=92)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q, dtype=torch.float64, device="cuda")
    _, F = ag.energy_and_forces(xt, qt, D, L, tol, precision="fp64", n_s=40)
    pot = ag.Potential("laplace", D, L, tol, precision="fp64", n_s=40)
    h = 1e-7
    frac = np.abs(x * 2 ** BITS - np.round(x * 2 ** BITS))       # distance to the nearest grid line
    cand = np.nonzero(np.min(frac, axis=1) > 4 * h * 2 ** BITS)[0]
    rng = np.random.default_rng(93)
    picks = rng.choice(cand, 12, replace=False)

    def energy(xx):
        u = pot(torch.tensor(xx, dtype=torch.float64, device="cuda"), qt.reshape(N, 1))
        return 0.5 * float((qt.reshape(N, 1) * u).sum())

    Fs = F.cpu().numpy()
    scale = np.sqrt(np.mean(np.sum(Fs ** 2, axis=1)))
    for t in picks:
        for i in range(3):
            xp, xm = x.copy(), x.copy()
            xp[t, i] += h
            xm[t, i] -= h
            fd = -(energy(xp) - energy(xm)) / (2 * h)
            assert abs(fd - Fs[t, i]) <= 10 * tol * scale + 1e-6 * abs(fd)
