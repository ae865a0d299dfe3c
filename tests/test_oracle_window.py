"""Pins of the oracle's PSWF window (Sec. 2.2) against its definition and scipy."""
import numpy as np
import pytest
import scipy.special as sp

from oracle.pswf import PSWFWindow
from oracle.params import TABLE


ALL_C = sorted({c for rows in TABLE.values() for (c, p) in rows})


@pytest.mark.parametrize("c", ALL_C)
def test_eigen_equation(c):
    """psi solves lambda psi(x) = int_{-1}^{1} psi(t) e^{ictx} dt (Eq. PSWFeig)."""
    w = PSWFWindow(c)
    t, wt = np.polynomial.legendre.leggauss(240)
    xs = np.linspace(-1, 1, 17)
    rhs = np.array([np.sum(wt * w.psi(t) * np.exp(1j * c * t * x)) for x in xs])
    lam = np.sum(wt * w.psi(t)) / w.psi0
    assert np.max(np.abs(rhs - lam * w.psi(xs))) <= 1e-13 * np.max(np.abs(rhs))
    # leading eigenfunction: no sign change on [-1, 1]
    assert np.all(w.psi(np.linspace(-1, 1, 2001)) > 0)


@pytest.mark.parametrize("c", [7.0, 10.47, 14.5])
def test_matches_scipy_prolate(c):
    w = PSWFWindow(c)
    xs = np.array([0.0, 0.1, 0.37, 0.6, 0.88, 0.99])
    ref = np.array([sp.pro_ang1(0, 0, c, x)[0] for x in xs])
    ref /= ref[0]
    assert np.allclose(w.psi(xs) / w.psi0, ref, rtol=1e-11, atol=0)


@pytest.mark.parametrize("c", [7.0, 14.5, 29.0])
def test_window_identities(c):
    """phi-hat(0)=1, Phi(0)=1, Phi(1)=0, and phi-hat is the Fourier transform of phi
    inside the band (Eqs. wfunchat_prop, def_erfc_like_fcn, wfunchat)."""
    w = PSWFWindow(c)
    assert abs(w.phihat(0.0) - 1) < 1e-15
    assert abs(w.Phi(0.0) - 1) < 1e-15
    assert abs(w.Phi(1.0 - 1e-16)) < 1e-13
    t, wt = np.polynomial.legendre.leggauss(240)
    for k in [0.0, 0.3 * c, 0.77 * c, c]:
        ft = np.sum(wt * w.phi(t) * np.cos(k * t))
        assert abs(ft - w.phihat(k)) < 1e-13
    # Phi' = -2 phi by finite differences
    r = np.linspace(0.05, 0.95, 7)
    h = 1e-6
    d = (w.Phi(r + h) - w.Phi(r - h)) / (2 * h)
    assert np.allclose(d, -2 * w.phi(r), atol=1e-7)


def test_gammaB_is_hasimoto_for_gaussian():
    """gammaB-hat = phi-hat - k phi-hat'/2 (Eq. gammaB_in_phi) gives Hasimoto's screening
    (1 + k^2/4) e^{-k^2/4} for the Gaussian phi-hat = e^{-k^2/4} (Sec. 1 and App. B)."""
    k = np.linspace(0, 6, 13)
    phihat = np.exp(-k * k / 4)
    dphihat = -k / 2 * phihat
    assert np.allclose(phihat - 0.5 * k * dphihat, (1 + k * k / 4) * np.exp(-k * k / 4), rtol=1e-15)
    # and the oracle's PSWF implementation of the same formula agrees with FD of phi-hat
    w = PSWFWindow(14.5)
    kk = np.linspace(0.5, 14.0, 9)
    h = 1e-6
    fd = (w.phihat(kk + h) - w.phihat(kk - h)) / (2 * h)
    assert np.allclose(w.gammaB_hat(kk), w.phihat(kk) - 0.5 * kk * fd, atol=1e-8)


def test_d2phihat0_by_fd():
    w = PSWFWindow(14.5)
    h = 1e-3
    fd = (w.phihat(h) - 2 * w.phihat(0.0) + w.phihat(-h)) / h ** 2
    assert abs(fd - w.d2phihat0()) < 1e-5 * abs(fd)
