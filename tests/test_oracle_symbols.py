"""Pins of the truncated-kernel symbols (Sec. 5.2, App. C) by quadrature of their
defining transforms, their printed kappa = 0 limits and the Lemma of App. C."""
import numpy as np
import pytest
import scipy.special as sp
from scipy.integrate import quad

from oracle import symbols as S

R = 2.0


def q(f, a, b):
    return quad(f, a, b, limit=400, epsabs=1e-14, epsrel=1e-13)[0]


@pytest.mark.parametrize("alpha,kappa", [(0.0, 0.0), (0.0, 0.7), (0.0, 5.3), (1.2, 0.0), (1.2, 2.5), (6.0, 4.0)])
def test_H1(alpha, kappa):
    """Eq. GreenR1D_Fourier = int_{-R}^{R} G_1^alpha(z) e^{-i kappa z} dz (Eq. Green1D)."""
    if alpha > 0:
        ref = q(lambda z: np.exp(-alpha * z) / alpha * np.cos(kappa * z), 0, R)
    else:
        ref = q(lambda z: -z * np.cos(kappa * z), 0, R)
    assert S.H1_trunc(alpha, kappa, R) == pytest.approx(ref, rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("alpha,kappa", [(0.0, 0.0), (0.0, 0.5), (0.0, 6.1), (1.1, 0.0), (1.1, 2.0), (5.0, 7.0)])
def test_H2(alpha, kappa):
    """Eq. GreenR2D_Fourier = 2 pi int_0^R J0(kappa r) G_2^alpha(r) r dr (Eq. radial_ft_2D) with
    G = K0(alpha r)/(2 pi), and for alpha = 0 the gauge -log(r/R)/(2 pi) that vanishes at R."""
    if alpha > 0:
        ref = q(lambda r: sp.k0(alpha * r) * sp.j0(kappa * r) * r, 0, R)
    else:
        ref = q(lambda r: -np.log(r / R) * sp.j0(kappa * r) * r, 0, R)
    assert S.H2_trunc(alpha, kappa, R) == pytest.approx(ref, rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("alpha,kappa", [(0.0, 0.0), (0.0, 0.9), (0.0, 4.4), (0.8, 0.0), (0.8, 3.0), (4.0, 1.5)])
def test_B1(alpha, kappa):
    """Eq. BGreenR1D_Fourier: alpha>0 from B = -(1/(2 alpha)) d/dalpha of e^{-alpha|z|}/(2 alpha)
    = e^{-alpha|z|}(alpha|z|+1)/(4 alpha^3); alpha = 0 the even C^1 gauge
    |z|^3/12 - R z^2/8 + R^3/24 vanishing with its slope at R."""
    if alpha > 0:
        f = lambda z: 2 * np.exp(-alpha * z) * (alpha * z + 1) / (4 * alpha ** 3) * np.cos(kappa * z)
    else:
        f = lambda z: 2 * (z ** 3 / 12 - R * z * z / 8 + R ** 3 / 24) * np.cos(kappa * z)
    assert S.B1_trunc(alpha, kappa, R) == pytest.approx(q(f, 0, R), rel=1e-10, abs=1e-13)


@pytest.mark.parametrize("kappa", [0.0, 0.6, 3.7])
def test_B2_zero_mode(kappa):
    """alpha = 0 of Eq. BGreenR2D_Fourier: the 2D biharmonic r^2(log r - 1)/(8 pi) in the gauge
    vanishing with its slope at R: + R^2/(16 pi) - (2 log R - 1) r^2/(16 pi)."""
    g = lambda r: r * r * (np.log(r) - 1) / (8 * np.pi) + R * R / (16 * np.pi) - (2 * np.log(R) - 1) * r * r / (16 * np.pi)
    ref = 2 * np.pi * q(lambda r: sp.j0(kappa * r) * g(r) * r, 0, R)
    assert S.B2_trunc(0.0, kappa, R) == pytest.approx(ref, rel=1e-10, abs=1e-13)


@pytest.mark.parametrize("d", [1, 2])
@pytest.mark.parametrize("alpha,kappa", [(0.7, 0.0), (0.7, 2.2), (3.1, 5.0)])
def test_lemma_biharmonic_from_harmonic(d, alpha, kappa):
    """Lemma biharmonic_from_harmonic: B-hat = -(1/(2 alpha)) d/dalpha H-hat (Eq. app_Bhat)."""
    H = S.H1_trunc if d == 1 else S.H2_trunc
    B = S.B1_trunc if d == 1 else S.B2_trunc
    h = 1e-5
    fd = (H(alpha + h, kappa, R) - H(alpha - h, kappa, R)) / (2 * h)
    assert B(alpha, kappa, R) == pytest.approx(-fd / (2 * alpha), rel=1e-7)


def test_printed_limits():
    """kappa = 0 values printed with Eqs. GreenR2D/1D_Fourier and BGreenR2D/1D_Fourier."""
    assert S.H2_trunc(0.0, 0.0, R) == R * R / 4
    assert S.H1_trunc(0.0, 0.0, R) == -R * R / 2
    assert S.B2_trunc(0.0, 0.0, R) == R ** 4 / 64
    assert S.B1_trunc(0.0, 0.0, R) == R ** 4 / 24
    for f, lim in [(lambda k: S.H2_trunc(0.0, k, R), R * R / 4), (lambda k: S.H1_trunc(0.0, k, R), -R * R / 2),
                   (lambda k: S.B2_trunc(0.0, k, R), R ** 4 / 64), (lambda k: S.B1_trunc(0.0, k, R), R ** 4 / 24)]:
        # continuity at kappa R = 0.02: the next Taylor term is O((kappa R)^2); smaller kappa
        # only adds cancellation in the closed forms (the discretisations never sample it:
        # free wavenumbers are n pi/R)
        assert f(0.01) == pytest.approx(lim, rel=1e-3)


@pytest.mark.parametrize("kappa", [0.0, 0.4, 2.0, 9.0])
def test_free_space_3d(kappa):
    """D=0: radial transform (Eq. radial_ft_3D) of 1/(4 pi r) truncated at R and of the C^1-gauge
    truncated biharmonic -r/(8 pi) + R/(16 pi) + r^2/(16 pi R)."""
    sinc = lambda r: np.sinc(kappa * r / np.pi)
    assert S.H3_trunc(kappa, R) == pytest.approx(q(lambda r: sinc(r) * r, 0, R), rel=1e-11)
    BR = lambda r: -r / (8 * np.pi) + R / (16 * np.pi) + r * r / (16 * np.pi * R)
    assert S.B3_trunc(kappa, R) == pytest.approx(4 * np.pi * q(lambda r: sinc(r) * BR(r) * r * r, 0, R),
                                                 rel=1e-9, abs=1e-13)


@pytest.mark.parametrize("k", [-3.0, 0.5, 2.0])
def test_Z1(k):
    """Eq. ZGreenR1D_Fourier = int_{-R}^{R} sgn(z)/4 e^{-ikz} dz."""
    ref = -1j * 2 * q(lambda z: np.sin(k * z) / 4, 0, R)
    assert S.Z1_trunc(k, R) == pytest.approx(ref, rel=1e-12)
