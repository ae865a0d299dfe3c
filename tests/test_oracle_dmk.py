"""Whole-pipeline pins of the oracle DMK (Sec. 3-5) against independent references.

* Laplace, every D: the Ewald-type reference of oracle/ewald.py (Gaussian split, no DMK
  machinery), to within the tolerance row (Table 2 reports errors below eps).
* D = 3: the NaCl Madelung constant (tests/golden/madelung_nacl.txt).
* Stokes kernels, D = 0: the O(N^2) free-space sum of App. B's kernels.
* Rotlet, D = 3, 2, 1: -1/2 curl of three Laplace potentials (Eq. rotlet_def_deriv).
* Stokeslet, D = 3, 2, 1: Hasimoto's Ewald split of the Oseen tensor (oracle/ewald.py; its
  smooth part checked against the inverse Fourier transform by quadrature, the slab's kappa_3
  integrals and the 2D angular means of D = 1 against quadrature), velocities and gradients.
* Stresslet, D = 3, 2, 1: the stress of the Stokeslet flow, T_jlm = -delta_jm P_l + d_m G_jl +
  d_j G_ml with the Stokeslet pressure P_l = -d_l (1/(4 pi r)), mode by mode for k != 0, so the
  periodic stresslet sum equals Stokeslet and Laplace gradient sums; the Stokeslet flows are
  divergence-free.
* Invariants: permutation, linearity, symmetry, periodic translation; 2:1 balance.
"""
import itertools
import os

import numpy as np
import pytest
from scipy.integrate import quad
import scipy.special as sp

from oracle.dmk import evaluate, evaluate_targets
from oracle import ewald
from oracle.kernels import Kernel
from oracle.params import Geometry
from oracle.tree import Forest, wrap_and_quantize, BITS

from paper_2606_27134_b300 import workloads


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


CASES = [(3, [1, 1, 1]), (3, [2, 1, 1]), (2, [1, 1, 0.5]), (2, [1, 2, 1]), (1, [1, 1, 1]), (1, [2, 1, 1]),
         (0, [1, 1, 1]),
         # non-exact tilings (Sec. 4.1.1-4.1.2: cut cubes, padding, source images): Table 2's
         # [1, 1.3, 1.7], the same with the padded axis first, and a slab with L_2 / L_1 = 1.3
         (3, [1, 1.3, 1.7]), (3, [1.3, 1, 1.7]), (2, [1, 1.3, 0.5]),
         # the other cells of Table 2: three cubes along a periodic axis with a free x3 of two,
         # five cubes along x2, and the singly periodic [3, 1, 2] and [1, 1, 2]
         (2, [3, 1, 2]), (2, [1, 5, 2]), (1, [3, 1, 2]), (1, [1, 1, 2])]


@pytest.mark.parametrize("D,L", CASES, ids=lambda v: str(v))
def test_laplace_vs_ewald(D, L):
    x, q = workloads.mixed_points(100, L, seed=11 + D), None
    q = workloads.neutral_charges(100, seed=5 + D)
    r = evaluate("laplace", D, L, 1e-6, x, q, n_s=12, grad=True)
    ue, ge = ewald.laplace_reference(D, L, x, q, grad=True)
    assert rel(r.u[:, 0], ue) < 1e-6
    assert rel(r.grad[:, :, 0], ge) < 3e-6


@pytest.mark.parametrize("L", [[1, 1, 1], [1, 1.3, 1.7]])
def test_laplace_vs_ewald_tight(L):
    """Table 2 reports 8.5e-11 for L = [1, 1.3, 1.7] at 1e-9 (a non-exact tiling)."""
    x = workloads.uniform_points(80, L, seed=3)
    q = workloads.neutral_charges(80, seed=4)
    r = evaluate("laplace", 3, L, 1e-9, x, q, n_s=10)
    assert rel(r.u[:, 0], ewald.laplace_reference(3, L, x, q)) < 1e-9


def _nacl(reps):
    a = 0.5
    pts, qs = [], []
    for i, j, k in itertools.product(range(2 * reps), repeat=3):
        pts.append([(i + 0.25) * a, (j + 0.25) * a, (k + 0.25) * a])
        qs.append((-1.0) ** (i + j + k))
    return np.array(pts), np.array(qs), [reps * 1.0] * 3, a


@pytest.mark.parametrize("reps", [1, 2])
def test_madelung(reps):
    M = float(open(os.path.join(os.path.dirname(__file__), "golden", "madelung_nacl.txt")).read().split()[-1])
    x, q, L, a = _nacl(reps)
    want = -q * M / (4 * np.pi * a)
    r = evaluate("laplace", 3, L, 1e-9, x, q, n_s=4)
    assert np.max(np.abs(r.u[:, 0] - want)) < 1e-9 * np.max(np.abs(want))
    assert np.max(np.abs(ewald.laplace_reference(3, L, x, q) - want)) < 1e-12


def test_ewald_2p_integral_closed_form():
    """The closed form used for the kappa_3 integral of Eq. ewald_far_2P_es (alpha > 0)."""
    nu = 0.3
    for alpha, z in [(2 * np.pi, 0.0), (2 * np.pi, 0.4), (8.9, -0.7), (20.0, 0.15)]:
        f = lambda k: np.exp(-(alpha ** 2 + k * k) * nu * nu / 4) / (alpha ** 2 + k * k) * np.cos(k * z)
        ref = 2 * quad(f, 0, np.inf, limit=400, epsabs=1e-15)[0]
        assert ewald._int_2p(alpha, z, nu) == pytest.approx(ref, rel=1e-10)
        h = 1e-6
        fd = (ewald._int_2p(alpha, z + h, nu) - ewald._int_2p(alpha, z - h, nu)) / (2 * h)
        assert ewald._dint_2p(alpha, z, nu) == pytest.approx(fd, rel=1e-6, abs=1e-10)
    # zero mode: int (e^{-k^2 nu^2/4} cos kz - 1)/k^2 dk
    for z in [0.1, 0.5, 1.3]:
        f = lambda k: (np.exp(-k * k * nu * nu / 4) * np.cos(k * z) - 1) / (k * k)
        K = 40.0 / nu                 # beyond K the Gaussian is < 1e-170; the -1/k^2 tail is -1/K
        ref = 2 * (quad(f, 0, K, limit=2000, epsabs=1e-14)[0] - 1.0 / K)
        # the reference drops the z-independent constant I(0) = -sqrt(pi) nu, which cancels
        # in sum_s q_s I(z_t - z_s) for neutral charges (the only case Sec. 5.2 admits)
        val = -np.pi * (z * sp.erf(z / nu) + nu / np.sqrt(np.pi) * (np.exp(-(z / nu) ** 2) - 1))
        assert val - np.sqrt(np.pi) * nu == pytest.approx(ref, rel=1e-8)


def test_ewald_1p_integrals():
    """Polar kappa integrals of Eq. ewald_far_1P_es: quadrature rule and the k1 = 0 closed form."""
    nu = 0.25
    rr = np.array([0.05, 0.3, 0.9])
    for k1 in [2 * np.pi, 4 * np.pi]:
        val, _ = ewald._polar_1p(k1, rr, nu)
        for i, r in enumerate(rr):
            f = lambda k: sp.j0(k * r) * np.exp(-(k1 ** 2 + k * k) * nu * nu / 4) / (k1 ** 2 + k * k) * k
            assert val[i] == pytest.approx(2 * np.pi * quad(f, 0, np.inf, limit=400)[0], rel=1e-9)
    for r in rr:
        f = lambda k: (sp.j0(k * r) - 1) * np.exp(-k * k * nu * nu / 4) / k
        ref = 2 * np.pi * quad(f, 0, np.inf, limit=400)[0]
        x = (r / nu) ** 2
        assert -np.pi * (sp.exp1(x) + np.log(x) + np.euler_gamma) == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet", "rotlet"])
def test_stokes_free_space_direct(kernel):
    """D = 0: oracle vs the O(N^2) sum of the kernels of App. B."""
    L = [1, 1, 1]
    N = 90
    x = workloads.mixed_points(N, L, seed=21)
    K = Kernel(kernel)
    rho = workloads.stokes_strengths(kernel, N, seed=22)
    r = evaluate(kernel, 0, L, 1e-6, x, rho, n_s=12, grad=True)
    dx = x[:, None, :] - x[None, :, :]
    ii, jj = np.nonzero(~np.eye(N, dtype=bool))
    Kv = K.full(dx[ii, jj])
    u = np.zeros((N, K.d_u))
    np.add.at(u, ii, np.einsum("nab,nb->na", Kv, rho[jj]))
    assert rel(r.u, u) < 2e-6
    # gradient by complex step of the direct sum
    g = np.zeros((N, 3, K.d_u))
    for i in range(3):
        d = dx[ii, jj].astype(complex)
        d[:, i] += 1e-30j
        gi = np.zeros((N, K.d_u), dtype=complex)
        np.add.at(gi, ii, np.einsum("nab,nb->na", K.full(d), rho[jj]))
        g[:, i, :] = gi.imag / 1e-30
    assert rel(r.grad, g) < 1e-5


@pytest.mark.parametrize("D,L", [(3, [1, 1, 1]), (2, [1, 1, 1]), (1, [1, 1, 1]), (3, [1, 1.3, 1.7])])
def test_rotlet_is_curl_of_laplace(D, L):
    """Eq. rotlet_def_deriv: Omega_jl tau_l = -1/2 eps_jlm d_m H tau_l, so the rotlet sum equals
    -1/2 curl of three Laplace potentials (one per torque component) -- to within eps."""
    N = 90
    x = workloads.mixed_points(N, L, seed=31)
    tau = workloads.stokes_strengths("rotlet", N, seed=32)
    tau -= tau.mean(axis=0)           # neutral components for the D < 3 Laplace sums
    r = evaluate("rotlet", D, L, 1e-9, x, tau, n_s=12)
    gl = np.stack([evaluate("laplace", D, L, 1e-9, x, tau[:, l], n_s=12, grad=True).grad[:, :, 0]
                   for l in range(3)], axis=1)          # gl[t, l, m] = d_m phi_l
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    want = -0.5 * np.einsum("jlm,tlm->tj", eps, gl)
    assert rel(r.u, want) < 1e-8


@pytest.mark.parametrize("r", [0.05, 0.3, 0.7, 1.5])
def test_hasimoto_smooth_part_is_inverse_transform(r):
    """G^F(x) of oracle/ewald.py equals (2 pi)^-3 int (I - k k^T/k^2) phi(k)/k^2 e^{ikx} d^3k,
    phi = (1 + k^2 nu^2/4) e^{-k^2 nu^2/4}, by radial quadrature: the angular mean of
    k_j k_l/k^2 e^{ikx} is j1(kr)/(kr) delta_jl - j2(kr) x_j x_l/r^2; and G^F(0) = I/(2 pi^1.5 nu)."""
    nu = 0.3
    xh = np.array([0.48, -0.6, 0.64])
    xh /= np.linalg.norm(xh)
    h = lambda k: (1 + k * k * nu * nu / 4) * np.exp(-k * k * nu * nu / 4)
    a = quad(lambda k: h(k) * (sp.spherical_jn(0, k * r) - sp.spherical_jn(1, k * r) / (k * r)), 0, 60 / nu,
             limit=500)[0] / (2 * np.pi ** 2)
    b = quad(lambda k: h(k) * sp.spherical_jn(2, k * r), 0, 60 / nu, limit=500)[0] / (2 * np.pi ** 2)
    want = a * np.eye(3) + b * np.outer(xh, xh)
    got = ewald.stokes_smooth((r * xh)[None], nu)[0]
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    self_q = quad(lambda k: h(k) * 2 / 3, 0, 60 / nu)[0] / (2 * np.pi ** 2)
    assert self_q == pytest.approx(1 / (2 * np.pi ** 1.5 * nu), rel=1e-12)
    small = ewald.stokes_smooth((1e-3 * xh)[None], nu)[0]
    assert np.abs(small - np.eye(3) / (2 * np.pi ** 1.5 * nu)).max() < 1e-5 / nu


@pytest.mark.parametrize("L", [[1, 1, 1], [1, 1, 2], [1, 1.3, 1.7]])
def test_stokeslet_3p_vs_ewald(L):
    """D = 3 Stokeslet: oracle vs Hasimoto's Ewald sum (two split parameters agree to roundoff),
    velocities and target gradients (complex step of the Ewald sum)."""
    N = 50
    x = workloads.mixed_points(N, L, seed=61)
    f = workloads.stokes_strengths("stokeslet", N, seed=62)
    r = evaluate("stokeslet", 3, L, 1e-9, x, f, n_s=12, grad=True)
    e1 = ewald.stokeslet_ewald_3p(x, x, f, L, 0.2 * min(L))
    e2 = ewald.stokeslet_ewald_3p(x, x, f, L, 0.3 * min(L))
    assert rel(e1, e2) < 1e-13
    assert rel(r.u, e1) < 1e-8
    h = 1e-20
    g = np.zeros((N, 3, 3))
    for i in range(3):
        xt = x.astype(complex)
        xt[:, i] += 1j * h
        g[:, i, :] = ewald.stokeslet_ewald_3p(xt, x, f, L, 0.25 * min(L)).imag / h
    assert rel(r.grad, g) < 1e-8


@pytest.mark.parametrize("alpha,z", [(2.0, 0.1), (5.0, -0.4), (9.0, 0.7), (0.8, 0.0)])
def test_stokes_slab_integrals(alpha, z):
    """The closed forms of the D = 2 Stokeslet reference: I0 = int phi/k^2 e^{ikz}, I2 =
    int phi/k^4 e^{ikz} and dI2/dz = -(z/2) I_L (k^2 = alpha^2 + kappa^2), by quadrature."""
    nu = 0.3
    phi = lambda k: (1 + (alpha ** 2 + k * k) * nu * nu / 4) * np.exp(-(alpha ** 2 + k * k) * nu * nu / 4)
    I0q = 2 * quad(lambda k: phi(k) / (alpha ** 2 + k * k) * np.cos(k * z), 0, 80 / nu, limit=400)[0]
    I2q = 2 * quad(lambda k: phi(k) / (alpha ** 2 + k * k) ** 2 * np.cos(k * z), 0, 80 / nu, limit=400)[0]
    dI2q = -2 * quad(lambda k: k * phi(k) / (alpha ** 2 + k * k) ** 2 * np.sin(k * z), 0, 80 / nu, limit=400)[0]
    I0, I2, IL = ewald._stokes_2p_modes(alpha, z, nu)
    assert I0 == pytest.approx(I0q, rel=1e-11)
    assert I2 == pytest.approx(I2q, rel=1e-11)
    assert -z / 2 * IL == pytest.approx(dI2q, rel=1e-10, abs=1e-14)


@pytest.mark.parametrize("L", [[1, 1, 1], [2, 1, 0.5]])
def test_stokeslet_2p_vs_ewald(L):
    """D = 2 Stokeslet (forces summing to zero): oracle vs the Ewald sum of oracle/ewald.py
    (two split parameters agree to roundoff), velocities and target gradients."""
    N = 50
    x = workloads.mixed_points(N, L, seed=71, D=2)
    f = workloads.stokes_strengths("stokeslet", N, seed=72)
    r = evaluate("stokeslet", 2, L, 1e-9, x, f, n_s=12, grad=True)
    s0 = 0.2 * min(L[:2])
    e1 = ewald.stokeslet_ewald_2p(x, x, f, L, s0)
    e2 = ewald.stokeslet_ewald_2p(x, x, f, L, 1.5 * s0)
    assert rel(e1, e2) < 1e-13
    assert rel(r.u, e1) < 1e-8
    h = 1e-20
    g = np.zeros((N, 3, 3))
    for i in range(3):
        xt = x.astype(complex)
        xt[:, i] += 1j * h
        g[:, i, :] = ewald.stokeslet_ewald_2p(xt, x, f, L, 1.25 * s0).imag / h
    assert rel(r.grad, g) < 1e-8


def test_polar_angular_means():
    """The 2D angular means the D = 1 Stokeslet reference uses, by quadrature over the angle:
    <q_a e^{iq.rho}> = i kappa J1 rhohat_a and <q_a q_b e^{iq.rho}> = kappa^2/2 [(J0 + J2) delta_ab
    - 2 J2 rhohat_a rhohat_b]."""
    kappa, rho = 3.7, np.array([0.21, -0.35])
    r = np.linalg.norm(rho)
    rh = rho / r
    th = np.linspace(0, 2 * np.pi, 4001)[:-1]
    q = kappa * np.stack([np.cos(th), np.sin(th)], -1)
    e = np.exp(1j * q @ rho)
    m1 = (q * e[:, None]).mean(axis=0)
    m2 = np.einsum("na,nb,n->ab", q, q, e) / len(th)
    J0, J1, J2 = (sp.jv(v, kappa * r) for v in (0, 1, 2))
    assert np.abs(m1 - 1j * kappa * J1 * rh).max() < 1e-12
    want = kappa ** 2 / 2 * ((J0 + J2) * np.eye(2) - 2 * J2 * np.outer(rh, rh))
    assert np.abs(m2 - want).max() < 1e-12


@pytest.mark.parametrize("L", [[1, 1, 1], [2, 1, 1]])
def test_stokeslet_1p_vs_ewald(L):
    """D = 1 Stokeslet (forces summing to zero): oracle vs the Ewald sum of oracle/ewald.py
    (two split parameters agree to roundoff), velocities and target gradients (complex step of
    1e-6: the complex Bessel routines are accurate relative to the function's size only)."""
    N = 40
    x = workloads.mixed_points(N, L, seed=81, D=1)
    f = workloads.stokes_strengths("stokeslet", N, seed=82)
    r = evaluate("stokeslet", 1, L, 1e-9, x, f, n_s=12, grad=True)
    s0 = 0.2 * L[0]
    e1 = ewald.stokeslet_ewald_1p(x, x, f, L, s0)
    e2 = ewald.stokeslet_ewald_1p(x, x, f, L, 1.5 * s0)
    assert rel(e1, e2) < 1e-13
    assert rel(r.u, e1) < 1e-8
    h = 1e-6
    g = np.zeros((N, 3, 3))
    for i in range(3):
        xt = x.astype(complex)
        xt[:, i] += 1j * h
        g[:, i, :] = ewald.stokeslet_ewald_1p(xt, x, f, L, 1.25 * s0).imag / h
    assert rel(r.grad, g) < 1e-8


@pytest.mark.parametrize("D,L", [(3, [1, 1, 1]), (2, [1, 1, 0.5]), (1, [1, 1, 1]), (3, [2, 1.3, 1.7])])
def test_stresslet_is_stokeslet_stress(D, L):
    """Stresslet (rho[s, 3l+m] = Q_lm) = sum_m [d_m u^(m)_j + d_j u^(m)_m] + sum_l d_l phi^(lj),
    u^(m) the Stokeslet velocity of the forces Q_lm (l = 0..2), phi^(lj) the Laplace potential of
    the charges Q_lj; every sum without its k = 0 mode.  For D < 3 every component of Q has zero
    sum, so that each Laplace and Stokeslet sum is defined.  Checked first in free space on the
    kernels themselves.  The Stokeslet flows are divergence-free: sum_j d_j u^(m)_j = 0."""
    KL, KG, KT = Kernel("laplace"), Kernel("stokeslet"), Kernel("stresslet")
    x0 = np.array([0.31, -0.52, 0.17])
    hh = 1e-6
    dG = np.zeros((3, 3, 3))
    P = np.zeros(3)
    for m in range(3):
        e = np.zeros(3)
        e[m] = hh
        dG[m] = (KG.full((x0 + e)[None])[0] - KG.full((x0 - e)[None])[0]) / (2 * hh)
        P[m] = -(KL.full((x0 + e)[None])[0, 0, 0] - KL.full((x0 - e)[None])[0, 0, 0]) / (2 * hh)
    Tc = np.zeros((3, 3, 3))
    for j, l, m in itertools.product(range(3), repeat=3):
        Tc[j, l, m] = -(j == m) * P[l] + dG[m, j, l] + dG[j, m, l]
    assert np.abs(KT.full(x0[None])[0] - Tc.reshape(3, 9)).max() < 1e-8 * np.abs(Tc).max()
    N, tol = 60, 1e-8
    x = workloads.mixed_points(N, L, seed=51, D=D)
    Q = workloads.stokes_strengths("stresslet", N, seed=52)
    if D < 3:
        Q = Q - Q.mean(axis=0)
    uT = evaluate("stresslet", D, L, tol, x, Q, n_s=12).u
    want = np.zeros((N, 3))
    for m in range(3):
        g = evaluate("stokeslet", D, L, tol, x, Q[:, [3 * l + m for l in range(3)]], n_s=12, grad=True).grad
        want += g[:, m, :] + g[:, :, m]
        assert np.linalg.norm(np.einsum("tjj->t", g)) < 1e-8 * np.linalg.norm(g)
    for l, j in itertools.product(range(3), repeat=2):
        want[:, j] += evaluate("laplace", D, L, tol, x, Q[:, 3 * l + j], n_s=12, grad=True).grad[:, l, 0]
    assert rel(uT, want) < 1e-8


def test_invariants():
    L = [1, 1, 1]
    N = 120
    x = workloads.uniform_points(N, L, seed=41)
    q = workloads.neutral_charges(N, seed=42)
    q2 = workloads.neutral_charges(N, seed=43)
    base = evaluate("laplace", 3, L, 1e-6, x, q, n_s=15).u[:, 0]
    perm = np.random.default_rng(0).permutation(N)
    up = evaluate("laplace", 3, L, 1e-6, x[perm], q[perm], n_s=15).u[:, 0]
    assert np.max(np.abs(up - base[perm])) < 1e-12 * np.max(np.abs(base))
    lin = evaluate("laplace", 3, L, 1e-6, x, 2 * q - 3 * q2, n_s=15).u[:, 0]
    b2 = evaluate("laplace", 3, L, 1e-6, x, q2, n_s=15).u[:, 0]
    assert np.max(np.abs(lin - (2 * base - 3 * b2))) < 1e-12 * np.max(np.abs(lin))
    # symmetry of the (symmetric) operator: q2 . u(q) = q . u(q2), to within eps
    assert abs(q2 @ base - q @ b2) < 1e-6 * np.sqrt(np.sum(base ** 2) * np.sum(q2 ** 2))
    # translation by a vector in the periodic directions (the tree changes; result within eps)
    shift = np.array([0.3137, -0.271, 0.5])
    ut = evaluate("laplace", 3, L, 1e-6, x + shift, q, n_s=15).u[:, 0]
    assert rel(ut, base) < 2e-6
    # a point moved by a whole period is the same point
    x3 = x.copy()
    x3[7, 0] += 1.0
    x3[9, 2] -= 1.0
    u3 = evaluate("laplace", 3, L, 1e-6, x3, q, n_s=15).u[:, 0]
    assert np.max(np.abs(u3 - base)) < 1e-12 * np.max(np.abs(base))


def test_tree_is_balanced():
    """Sec. 3.1.1: leaves hold <= n_s points and touching leaves differ by at most one level."""
    geom = Geometry(3, [1, 1, 1])
    x = workloads.clustered_points(600, [1, 1, 1], seed=51, n_centers=3, sigma=0.02)
    w, G = wrap_and_quantize(x, geom)
    f = Forest(geom, G, 10)
    leaves = f.leaves()
    assert all(len(b.pts) <= 10 for b in leaves)
    assert sum(len(b.pts) for b in leaves) == len(x)
    n = 2 ** BITS
    for a in leaves:
        for b in leaves:
            if b.level < a.level + 2:
                continue
            for sh in itertools.product((-1, 0, 1), repeat=3):
                ok = True
                for i in range(3):
                    alo, ahi = a.ix[i] << (BITS - a.level), (a.ix[i] + 1) << (BITS - a.level)
                    blo, bhi = (b.ix[i] << (BITS - b.level)) + sh[i] * n, ((b.ix[i] + 1) << (BITS - b.level)) + sh[i] * n
                    ok &= blo <= ahi and alo <= bhi
                assert not ok


def test_gradient_is_derivative():
    """Complex-step gradient == central difference of the oracle's own u(x_t).

    The moved point carries zero strength, so u_t depends on x_t only as a target, and
    it stays far from every integer grid line (the tree does not change).
    """
    L = [1, 1, 1]
    N = 60
    x = workloads.uniform_points(N, L, seed=61)
    q = workloads.neutral_charges(N, seed=62)
    h = 1e-7
    frac = np.abs(x * 2 ** BITS - np.round(x * 2 ** BITS))
    t = int(np.argmax(np.min(frac, axis=1)))
    assert np.min(frac[t]) > 4 * h * 2 ** BITS
    q[t] = 0.0
    r = evaluate("laplace", 3, L, 1e-6, x, q, n_s=10, grad=True)
    for i in range(3):
        xp, xm = x.copy(), x.copy()
        xp[t, i] += h
        xm[t, i] -= h
        up = evaluate("laplace", 3, L, 1e-6, xp, q, n_s=10).u[t, 0]
        um = evaluate("laplace", 3, L, 1e-6, xm, q, n_s=10).u[t, 0]
        assert (up - um) / (2 * h) == pytest.approx(r.grad[t, i, 0], rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("kernel,D,L", [("laplace", 2, [1, 1, 0.5]), ("stokeslet", 1, [2, 1, 1])])
def test_target_subset_equals_full(kernel, D, L):
    """Restricting the leaf step to a subset of targets returns, for those targets, the values
    of the full evaluation (same forest, far field and residual sums; only the order in which
    numpy contracts the Chebyshev sums may differ, hence 1e-14 and not bitwise), and NaN
    elsewhere."""
    N = 500
    x = workloads.mixed_points(N, L, seed=31, D=D)
    rho = workloads.stokes_strengths(kernel, N, seed=32) if kernel != "laplace" else \
        workloads.neutral_charges(N, seed=32).reshape(N, 1)
    full = evaluate(kernel, D, L, 1e-6, x, rho, n_s=20, grad=True)
    idx = np.random.default_rng(33).choice(N, 60, replace=False)
    sub = evaluate(kernel, D, L, 1e-6, x, rho, n_s=20, grad=True, targets=idx)
    assert rel(sub.u[idx], full.u[idx]) < 1e-14
    assert rel(sub.grad[idx], full.grad[idx]) < 1e-14
    rest = np.setdiff1d(np.arange(N), idx)
    assert np.all(np.isnan(sub.u[rest])) and np.all(np.isnan(sub.grad[rest]))


@pytest.mark.parametrize("kernel,D,L,N,parts", [
    ("laplace", 3, [1, 1, 6], 900, [[0, 1, 2], [3, 4, 5]]),
    # free axis: the truncated-kernel constant multiplies the total strength (Remark
    # stokeslet_const_corr), which only the reduction supplies
    ("stokeslet", 1, [1, 1, 4], 500, [[0, 3], [1, 2]]),
])
def test_split_over_cubes_equals_full(kernel, D, L, N, parts):
    """The structure factor of Eq. structurefac is a sum over the cubes and the near field of a
    target reaches only the adjacent cubes: two evaluators, each given its own cubes' points
    plus those of the adjacent cubes, each summing chi (and the total strength) over its own
    cubes, the partial sums added, reproduce the full evaluation at their own targets (to
    rounding)."""
    from oracle.params import Geometry
    from oracle.tree import BITS, quantize, wrap
    tol = 1e-6
    d = 3 if kernel == "stokeslet" else 1
    x = workloads.uniform_points(N, L, seed=61)
    # Stokeslet forces with a net force, so that the constant is not zero
    q = (workloads.neutral_charges(N, seed=62).reshape(N, 1) if d == 1
         else np.random.default_rng(62).standard_normal((N, 3)) + 0.5)
    full = evaluate(kernel, D, L, tol, x, q, n_s=40, grad=True)
    geom = Geometry(D, L)
    M = geom.M
    Gc = quantize(wrap(x, geom), geom) >> BITS
    cube = Gc[:, 0] + M[0] * (Gc[:, 1] + M[1] * Gc[:, 2])
    ix = lambda m: np.array([m % M[0], (m // M[0]) % M[1], m // (M[0] * M[1])])

    def near(a, b):
        da = np.abs(ix(a) - ix(b))
        for i in range(3):
            if geom.periodic[i]:
                da[i] = min(da[i], M[i] - da[i])
        return np.all(da <= 1)

    ncube = M[0] * M[1] * M[2]
    keeps = []
    for own in parts:
        ghost = {m for m in range(ncube) for o in own if near(m, o)}
        keeps.append(np.isin(cube, sorted(set(own) | ghost)))
    partial = {}
    for rank, own in enumerate(parts):
        # the first pass only records this evaluator's partial sums
        keep = keeps[rank]
        evaluate(kernel, D, L, tol, x[keep], q[keep], n_s=40, owned_cubes=own,
                 chi_reduce=lambda c, r=rank: partial.__setitem__(r, c.copy()) or c,
                 targets=np.nonzero(np.isin(cube[keep], own))[0])
    total = partial[0] + partial[1]
    u = np.full(full.u.shape, np.nan)
    g = np.full(full.grad.shape, np.nan)
    for rank, own in enumerate(parts):
        keep = keeps[rank]
        idx = np.nonzero(keep)[0]
        mine = np.nonzero(np.isin(cube[keep], own))[0]
        r = evaluate(kernel, D, L, tol, x[keep], q[keep], n_s=40, grad=True, owned_cubes=own,
                     chi_reduce=lambda c: total, targets=mine)
        u[idx[mine]] = r.u[mine]
        g[idx[mine]] = r.grad[mine]
    assert rel(u, full.u) < 1e-13
    assert rel(g, full.grad) < 1e-13


@pytest.mark.parametrize("D,L", [(3, [1, 1, 1]), (2, [1, 1, 0.5]), (1, [1.5, 1, 1]), (3, [1, 1.3, 1.7])])
def test_separate_targets_laplace_vs_ewald(D, L):
    """Targets apart from the sources (evaluate_targets) against the Ewald sum of the sources
    at those points (an Ewald sum over sources and targets with the targets' strengths zero)."""
    N, M = 90, 60
    x = workloads.mixed_points(N, L, seed=401 + D)
    q = workloads.neutral_charges(N, seed=402 + D)
    y = workloads.uniform_points(M, L, seed=403 + D)

    r = evaluate_targets("laplace", D, L, 1e-6, x, q, y, n_s=12, grad=True)
    ue, ge = ewald.laplace_reference(D, L, np.vstack([y, x]), np.concatenate([np.zeros(M), q]), grad=True)
    assert r.u.shape == (M, 1)
    assert rel(r.u[:, 0], ue[:M]) < 1e-6
    assert rel(r.grad[:, :, 0], ge[:M]) < 3e-6


def test_separate_targets_stokeslet_3p_vs_ewald():
    """Stokeslet, D = 3, targets apart from the sources, against Hasimoto's Ewald sum."""
    L = [1, 1, 1]
    x = workloads.mixed_points(50, L, seed=411)
    f = workloads.stokes_strengths("stokeslet", 50, seed=412)
    y = workloads.uniform_points(30, L, seed=413)
    r = evaluate_targets("stokeslet", 3, L, 1e-9, x, f, y, n_s=12)
    # the Ewald sum's target t is its source t: sources and targets joined, target forces zero
    pts = np.vstack([y, x])
    e = ewald.stokeslet_ewald_3p(pts, pts, np.vstack([np.zeros((30, 3)), f]), L, 0.25)[:30]
    assert rel(r.u, e) < 1e-8


@pytest.mark.parametrize("D,L,tol", [(2, [1, 1, 4], 1e-6), (1, [1, 4, 4], 1e-6), (2, [1, 1, 1], 1e-3),
                                     (1, [1, 1, 1], 1e-3)])
def test_original_symbol_switch_vs_ewald(D, L, tol):
    """With the App. E switch on (original symbol on the step-pi/L_j grid for alpha != 0,
    truncated zero modes on the step-pi/R grid, Sec. 5.3) the Laplace sum stays within the
    tolerance of the Ewald sum."""
    from oracle.params import Geometry, original_symbol_ok
    assert original_symbol_ok("laplace", Geometry(D, L), tol)
    N = 80
    x = workloads.mixed_points(N, L, seed=431 + D)
    q = workloads.neutral_charges(N, seed=432 + D)
    r = evaluate("laplace", D, L, tol, x, q, n_s=12, grad=True)
    assert r.plan["nparts"] == 2
    ue, ge = ewald.laplace_reference(D, L, x, q, grad=True)
    assert rel(r.u[:, 0], ue) < tol
    assert rel(r.grad[:, :, 0], ge) < 3 * tol


@pytest.mark.parametrize("D,L", [(2, [1, 1, 3]), (1, [1, 3, 3])])
def test_original_symbol_switch_stokeslet_vs_ewald(D, L):
    """The same for the Stokeslet (m = 2 estimate) against Hasimoto's split, at 1e-9."""
    from oracle.params import Geometry, original_symbol_ok
    assert original_symbol_ok("stokeslet", Geometry(D, L), 1e-9)
    N = 40
    x = workloads.mixed_points(N, L, seed=441 + D, D=D)
    f = workloads.stokes_strengths("stokeslet", N, seed=442 + D)
    r = evaluate("stokeslet", D, L, 1e-9, x, f, n_s=12)
    assert r.plan["nparts"] == 2
    e = (ewald.stokeslet_ewald_2p if D == 2 else ewald.stokeslet_ewald_1p)(x, x, f, L, 0.2 * L[0])
    assert rel(r.u, e) < 1e-8


@pytest.mark.parametrize("D,L", [(3, [1, 1, 1]), (2, [1, 1, 1]), (1, [2, 1, 1])])
def test_stresslet_adjoint_identity(D, L):
    """The periodized stresslet T_jlm = -delta_jm P_l + d_m G_jl + d_j G_ml is fully symmetric
    in (j, l, m) and odd, so for any Q and g: sum_t g_t . u[Q]_t = -sum_m <Q[:, :, m],
    S[g (x) e_m]> -- the identity behind the stresslet's vector-Jacobian product.  The method's
    discretised operator keeps it to rounding."""
    N = 60
    x = workloads.uniform_points(N, L, seed=5)
    rng = np.random.default_rng(6)
    Q = rng.standard_normal((N, 9))
    g = rng.standard_normal((N, 3))
    lhs = np.sum(g * evaluate("stresslet", D, L, 1e-9, x, Q, n_s=12).u)
    rhs = 0.0
    for m in range(3):
        Qm = np.zeros((N, 3, 3))
        Qm[:, :, m] = g
        rhs -= np.sum(Q.reshape(N, 3, 3)[:, :, m] * evaluate("stresslet", D, L, 1e-9, x, Qm.reshape(N, 9), n_s=12).u)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
