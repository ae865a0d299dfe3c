"""Fourier symbols of the truncated Green's functions (oracle; test infrastructure only).

Sec. 5.2 (Eqs. GreenR2D_Fourier, GreenR1D_Fourier) for the harmonic kernel,
App. C (Eqs. BGreenR2D_Fourier, BGreenR1D_Fourier, ZGreenR1D_Fourier) for the
biharmonic and sign-function kernels, and the radial transform of App. A
(Eq. radial_ft_3D) for the free-space (D=0) truncated kernel.  Bessel functions
come from scipy.special.  Every function is vectorised over kappa; alpha is a
scalar or an array broadcastable against kappa.
"""
import numpy as np
import scipy.special as sp


def _bcast(alpha, kappa):
    a = np.asarray(alpha, dtype=np.float64)
    k = np.asarray(kappa, dtype=np.float64)
    return np.broadcast_arrays(a, k)


def H1_trunc(alpha, kappa, R):
    """Harmonic kernel, one free direction, truncated at |z|<=R (Eq. GreenR1D_Fourier)."""
    a, k = _bcast(alpha, kappa)
    k = np.abs(k)
    out = np.empty(a.shape)
    nz = a > 0
    e = np.exp(-a[nz] * R)
    kk = k[nz]
    out[nz] = (1 - e * np.cos(kk * R) + kk * e * np.sin(kk * R) / a[nz]) / (a[nz] ** 2 + kk ** 2)
    z = ~nz
    k0 = k[z]
    with np.errstate(invalid="ignore", divide="ignore"):
        v = (1 - R * k0 * np.sin(k0 * R) - np.cos(k0 * R)) / k0 ** 2
    out[z] = np.where(k0 > 0, v, -R * R / 2)
    return out


def H2_trunc(alpha, kappa, R):
    """Harmonic kernel, two free directions, truncated at |r|<=R (Eq. GreenR2D_Fourier)."""
    a, k = _bcast(alpha, kappa)
    out = np.empty(a.shape)
    nz = a > 0
    an, kn = a[nz], k[nz]
    out[nz] = (1 + kn * R * sp.j1(kn * R) * sp.k0(an * R)
               - an * R * sp.j0(kn * R) * sp.k1(an * R)) / (an ** 2 + kn ** 2)
    z = ~nz
    k0 = k[z]
    with np.errstate(invalid="ignore", divide="ignore"):
        v = (1 - sp.j0(R * k0)) / k0 ** 2
    out[z] = np.where(k0 > 0, v, R * R / 4)
    return out


def B1_trunc(alpha, kappa, R):
    """Biharmonic kernel, one free direction (Eq. BGreenR1D_Fourier)."""
    a, k = _bcast(alpha, kappa)
    k = np.abs(k)
    out = np.empty(a.shape)
    nz = a > 0
    an, kn = a[nz], k[nz]
    e = np.exp(-an * R)
    s2 = an ** 2 + kn ** 2
    out[nz] = (2 * an ** 3 + kn * e * (an * R * s2 + 3 * an ** 2 + kn ** 2) * np.sin(kn * R)
               - an ** 2 * e * (R * s2 + 2 * an) * np.cos(kn * R)) / (2 * an ** 3 * s2 ** 2)
    z = ~nz
    k0 = k[z]
    with np.errstate(invalid="ignore", divide="ignore"):
        v = (1 - np.cos(k0 * R) - k0 * R * np.sin(k0 * R) / 2) / k0 ** 4
    out[z] = np.where(k0 > 0, v, R ** 4 / 24)
    return out


def B2_trunc(alpha, kappa, R):
    """Biharmonic kernel, two free directions (Eq. BGreenR2D_Fourier)."""
    a, k = _bcast(alpha, kappa)
    out = np.empty(a.shape)
    nz = a > 0
    an, kn = a[nz], k[nz]
    s2 = an ** 2 + kn ** 2
    K0, K1 = sp.k0(an * R), sp.k1(an * R)
    J0, J1 = sp.j0(kn * R), sp.j1(kn * R)
    out[nz] = (1 - R * J0 * (R * s2 * K0 + 2 * an * K1) / 2
               + kn * R * J1 * (R * s2 * K1 / (2 * an) + K0)) / s2 ** 2
    z = ~nz
    k0 = k[z]
    with np.errstate(invalid="ignore", divide="ignore"):
        v = (1 - sp.j0(k0 * R) - k0 * R * sp.j1(k0 * R) / 2) / k0 ** 4
    out[z] = np.where(k0 > 0, v, R ** 4 / 64)
    return out


def Z1_trunc(kappa3, R):
    """Truncated sign-function kernel sgn(x)/4 (Eq. ZGreenR1D_Fourier); odd, signed kappa."""
    k = np.asarray(kappa3, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        v = -1j * (1 - np.cos(k * R)) / (2 * k)
    return np.where(k != 0, v, 0.0 + 0.0j)


def H3_trunc(kappa, R):
    """Free-space harmonic kernel 1/(4 pi r) truncated at r<=R, from Eq. radial_ft_3D:
    4 pi int_0^R sin(kr)/(kr) r^2/(4 pi r) dr = (1 - cos kR)/k^2, R^2/2 at k=0."""
    k = np.asarray(kappa, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        v = (1 - np.cos(k * R)) / k ** 2
    return np.where(k > 0, v, R * R / 2)


def B3_trunc(kappa, R):
    """Free-space biharmonic kernel truncated at r <= R, in a C^1 gauge.

    The paper gives no D=0 formula (Sec. 3.1.3 defers to Vico et al.).  Reading, by analogy
    with App. C (where the gauge freedom of the biharmonic Green's function is used so the
    truncated kernel vanishes with C^1 regularity and keeps the decay of the original):
        B_R(r) = -r/(8 pi) + R/(16 pi) + r^2/(16 pi R)  for r <= R, 0 beyond,
    which vanishes with its slope at R.  The added quadratic is biharmonic; the Stokeslet
    operator maps it to the constant -I/(4 pi R) (corrected after the root sum), the
    stresslet operator (third derivatives) to zero.  Transform by Eq. radial_ft_3D:
        (4 pi/k) int_0^R r sin(kr) B_R(r) dr,  limit at k = 0:  R^4 / 60 ... evaluated below.
    """
    k = np.asarray(kappa, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        kR = k * R
        s, c = np.sin(kR), np.cos(kR)
        I1 = (s - kR * c) / k ** 2                                            # int r sin
        I2 = (2 * kR * s + (2 - kR ** 2) * c - 2) / k ** 3                    # int r^2 sin
        I3 = (3 * (kR ** 2 - 2) * s - kR * (kR ** 2 - 6) * c) / k ** 4        # int r^3 sin
        v = 4 * np.pi / k * (-I2 / (8 * np.pi) + R * I1 / (16 * np.pi) + I3 / (16 * np.pi * R))
    # k -> 0: 4 pi int_0^R r^2 B_R(r) dr = 4 pi R^4 (-1/32 + 1/48 + 1/80)/pi
    lim = 4 * R ** 4 * (-1.0 / 32 + 1.0 / 48 + 1.0 / 80)
    return np.where(k > 0, v, lim)


def stokeslet_free_space_constant(R):
    """Constant the C^1 gauge of B3_trunc removes from the Stokeslet: + I/(4 pi R) per unit force."""
    return 1.0 / (4 * np.pi * R)
