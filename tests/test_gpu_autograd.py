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
    assert torch.allclose(gq, u.detach(), rtol=1e-9, atol=1e-12 * float(u.detach().abs().max()))


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


def test_forces_finite_difference_fullsize_clusters():
    """The adaptive workload at full size (N = 1e6 points in 64 Gaussian clusters, sigma 0.02,
    balanced +-1 charges, D = 3, tol 1e-6), plain FP64 path, fixed tree: forces through autograd
    (dmk_vjp) on a 1000-point subset (seed 2005) against central differences of the energy.
    Moving the whole subset at once along random directions v gives the directional derivative
    sum_a F_a . v_a from two evaluations; a few dozen single-coordinate differences follow.
    Only points farther than 4h from every line of the finest integer grid are moved, so every
    point keeps its integer coordinates and the forest is the same for all evaluations."""
    N, L, D, tol, h = 1_000_000, [1.0, 1.0, 1.0], 3, 1e-6, 1e-7
    x = W.clustered_points(N, L, 2005, n_centers=64, sigma=0.02)
    q = W.balanced_charges(N, 2006)
    frac = np.abs(x * 2 ** BITS - np.round(x * 2 ** BITS))
    cand = np.nonzero(np.min(frac, axis=1) > 4 * h * 2 ** BITS)[0]
    rng = np.random.default_rng(2005)
    sub = rng.choice(cand, 1000, replace=False)
    dev = torch.device("cuda", 0)
    xt = torch.tensor(x, dtype=torch.float64, device=dev)
    qt = torch.tensor(q, dtype=torch.float64, device=dev).reshape(N, 1)
    pot = ag.Potential("laplace", D, L, tol, precision="fp64", n_s=250)
    xg = xt.clone().requires_grad_(True)
    u = pot(xg, qt)
    E = 0.5 * (qt * u).sum()
    (gx,) = torch.autograd.grad(E, xg)
    F = -gx[torch.tensor(sub, device=dev)].cpu().numpy()
    nb0 = pot.plan.stats()["n_boxes"]

    def energy(dx):
        xx = xt.clone()
        xx[torch.tensor(sub, device=dev)] += torch.tensor(dx, dtype=torch.float64, device=dev)
        with torch.no_grad():
            uu = pot(xx, qt)
        assert pot.plan.stats()["n_boxes"] == nb0
        return 0.5 * float((qt * uu).sum())

    scale = np.linalg.norm(F)
    for k in range(4):
        v = rng.standard_normal((1000, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        fd = -(energy(h * v) - energy(-h * v)) / (2 * h)
        an = float(np.sum(F * v))
        assert abs(fd - an) <= 10 * tol * scale, (k, fd, an)
    fscale = np.sqrt(np.mean(np.sum(F ** 2, axis=1)))
    for a in rng.choice(1000, 8, replace=False):
        for i in range(3):
            e = np.zeros((1000, 3))
            e[a, i] = h
            fd = -(energy(e) - energy(-e)) / (2 * h)
            assert abs(fd - F[a, i]) <= 10 * tol * fscale + 1e-6 * abs(fd), (a, i, fd, F[a, i])


@pytest.mark.parametrize("kernel,D,L", [("laplace", 2, [1.0, 1.0, 0.5]), ("laplace", 1, [1.0, 1.0, 1.0]),
                                        ("rotlet", 3, [1.0, 1.0, 1.0]), ("stokeslet", 2, [1.0, 1.0, 1.0])])
def test_vjp_nonneutral_upstream_gradient(kernel, D, L):
    """L = sum_t |u_t|^2 / 2: its upstream gradient g = u does not sum to zero.  dmk_vjp's
    position gradient against central differences of L (fixed tree), and its strength gradient
    against the change of L under a neutral change of the strengths (exact up to the constant
    that no neutral change sees)."""
    N, tol, h = 1200, 1e-6, 1e-7
    x = W.mixed_points(N, L, 95, D=D)
    rho = W.stokes_strengths(kernel, N, 96)
    dev = torch.device("cuda", 0)
    xt = torch.tensor(x, dtype=torch.float64, device=dev)
    rt = torch.tensor(rho, dtype=torch.float64, device=dev)
    pot = ag.Potential(kernel, D, L, tol, precision="fp64", n_s=40)

    def loss(xx, rr):
        uu = pot(xx, rr)
        return 0.5 * (uu * uu).sum()

    xg = xt.clone().requires_grad_(True)
    rg = rt.clone().requires_grad_(True)
    Lv = loss(xg, rg)
    gx, gr = torch.autograd.grad(Lv, (xg, rg))
    u0 = pot(xt, rt)
    assert abs(float(u0.sum(0).abs().max())) > 1e-3 * float(u0.abs().sum())   # g really is non-neutral
    gx, gr = gx.cpu().numpy(), gr.cpu().numpy()
    frac = np.abs(x * 2 ** BITS - np.round(x * 2 ** BITS))
    cand = np.nonzero(np.min(frac, axis=1) > 4 * h * 2 ** BITS)[0]
    rng = np.random.default_rng(97)
    fscale = np.sqrt(np.mean(np.sum(gx ** 2, axis=1)))
    with torch.no_grad():
        for a in rng.choice(cand, 4, replace=False):
            for i in range(3):
                xp, xm = xt.clone(), xt.clone()
                xp[a, i] += h
                xm[a, i] -= h
                fd = (float(loss(xp, rt)) - float(loss(xm, rt))) / (2 * h)
                assert abs(fd - gx[a, i]) <= 10 * tol * fscale + 1e-6 * abs(fd), (a, i, fd, gx[a, i])
        # neutral change of the strengths: +e at one point, -e at another
        d = np.zeros_like(rho)
        d[3] = 1.0
        d[11] = -1.0
        dt = torch.tensor(d, dtype=torch.float64, device=dev)
        eps = 1e-4
        fd = (float(loss(xt, rt + eps * dt)) - float(loss(xt, rt - eps * dt))) / (2 * eps)
        an = float(np.sum(gr * d))
        # the adjoint is one more evaluation of the eps-approximate sum: agreement to 10 tol
        assert abs(fd - an) <= 10 * tol * (np.abs(gr[3]).sum() + np.abs(gr[11]).sum()), (fd, an)


@pytest.mark.parametrize("D,L", [(3, [1.0, 1.0, 2.0]), (2, [1.0, 1.0, 1.0]), (1, [2.0, 1.0, 1.0])])
def test_stresslet_vjp(D, L):
    """The stresslet through autograd (dmk_vjp with three evaluations of strengths g (x) e_m).
    Strengths: u is linear in Q, so sum_t g_t . u[dQ]_t must equal <dL/dQ, dQ> for any dQ (the
    discretised operator keeps the kernel's symmetry: the oracle satisfies this to 1e-15).
    Positions: central differences of L (fixed tree, plain FP64 path)."""
    N, tol, h = 1000, 1e-6, 1e-7
    x = W.mixed_points(N, L, 195, D=D)
    Q = W.stokes_strengths("stresslet", N, 196)
    dev = torch.device("cuda", 0)
    xt = torch.tensor(x, dtype=torch.float64, device=dev)
    Qt = torch.tensor(Q, dtype=torch.float64, device=dev)
    g = torch.tensor(np.random.default_rng(197).standard_normal((N, 3)), dtype=torch.float64, device=dev)
    pot = ag.Potential("stresslet", D, L, tol, precision="fp64", n_s=40)

    def loss(xx, qq):
        return (g * pot(xx, qq)).sum()

    xg = xt.clone().requires_grad_(True)
    qg = Qt.clone().requires_grad_(True)
    gx, gq = torch.autograd.grad(loss(xg, qg), (xg, qg))
    with torch.no_grad():
        for seed in (198, 199):
            dQ = torch.tensor(np.random.default_rng(seed).standard_normal((N, 9)), dtype=torch.float64, device=dev)
            lhs = float((g * pot(xt, dQ)).sum())
            rhs = float((gq * dQ).sum())
            assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + float((gq.abs() * dQ.abs()).sum())), (lhs, rhs)
        gxn = gx.cpu().numpy()
        frac = np.abs(x * 2 ** BITS - np.round(x * 2 ** BITS))
        cand = np.nonzero(np.min(frac, axis=1) > 4 * h * 2 ** BITS)[0]
        fscale = np.sqrt(np.mean(np.sum(gxn ** 2, axis=1)))
        for a in np.random.default_rng(200).choice(cand, 4, replace=False):
            for i in range(3):
                xp, xm = xt.clone(), xt.clone()
                xp[a, i] += h
                xm[a, i] -= h
                fd = (float(loss(xp, Qt)) - float(loss(xm, Qt))) / (2 * h)
                assert abs(fd - gxn[a, i]) <= 10 * tol * fscale + 1e-6 * abs(fd), (a, i, fd, gxn[a, i])
