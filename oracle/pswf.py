"""Window functions for the kernel split (oracle; test infrastructure only).

Sec. 2.2: the window phi is even, phi-hat(0)=1, and Phi(r) = 1 - 2 int_0^r phi
(Eq. def_erfc_like_fcn).  The PSWF window (Eqs. PSWFeig, wfunc_pswf, wfunchat)
takes psi = psi_0^c, the leading eigenfunction of the band-limited Fourier
transform on [-1,1]; phi = psi / int psi, and phi-hat(k) = psi(k/c)/psi(0) for
|k| <= c, zero beyond (numerical truncation at the band limit).

Remark PSWF_eval: psi is evaluated through its Legendre expansion.  Here the
expansion coefficients come from the prolate differential operator
    L = -(d/dx)(1-x^2)(d/dx) + c^2 x^2,
which commutes with the finite Fourier transform of Eq. PSWFeig, so psi_0^c is
the eigenfunction of L with the smallest eigenvalue.  In the normalised
Legendre basis sqrt(n+1/2) P_n the operator is symmetric tridiagonal on the
even degrees (x^2 couples n to n and n+-2); a dense symmetric eigensolver
(numpy.linalg.eigh) gives the coefficients.

Biharmonic screening (App. B, Eq. gammaB_in_phi): gammaB-hat(k) = phi-hat(k) - k phi-hat'(k)/2.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


class PSWFWindow:
    """PSWF window with band limit c (Sec. 2.2)."""

    def __init__(self, c, n_even=None):
        self.c = float(c)
        if n_even is None:
            n_even = int(np.ceil(self.c)) + 40
        n = np.arange(0, 2 * n_even, 2, dtype=np.float64)
        c2 = self.c * self.c
        # <x^2 Pbar_n, Pbar_n> = (2n^2+2n-1)/((2n-1)(2n+3)),
        # <x^2 Pbar_n, Pbar_{n+2}> = (n+1)(n+2)/((2n+3) sqrt((2n+1)(2n+5)))
        diag = n * (n + 1) + c2 * (2 * n * n + 2 * n - 1) / ((2 * n - 1) * (2 * n + 3))
        m = n[:-1]
        off = c2 * (m + 1) * (m + 2) / ((2 * m + 3) * np.sqrt((2 * m + 1) * (2 * m + 5)))
        A = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
        evals, evecs = np.linalg.eigh(A)
        a = evecs[:, 0]
        coef = np.zeros(2 * n_even)
        coef[0::2] = a * np.sqrt(n + 0.5)          # standard Legendre coefficients of psi
        if npleg.legval(0.0, coef) < 0:
            coef = -coef
        self.chi0 = evals[0]
        self.psi_coef = coef
        self.psi0 = npleg.legval(0.0, coef)
        # int_{-1}^{1} psi = 2 * (P_0 coefficient)
        self.psi_int = 2.0 * coef[0]
        self.phi_coef = coef / self.psi_int                      # Eq. wfunc_pswf
        self.dpsi_coef = npleg.legder(coef)
        self.d2psi_coef = npleg.legder(coef, 2)
        self.dphi_coef = npleg.legder(self.phi_coef)
        # antiderivative of phi vanishing at 0, used by Phi (Eq. def_erfc_like_fcn)
        self.iphi_coef = npleg.legint(self.phi_coef, lbnd=0.0)

    # ---- real-space window -------------------------------------------------
    def psi(self, x):
        return npleg.legval(np.asarray(x, dtype=np.float64), self.psi_coef)

    def phi(self, x):
        """phi(x) = psi(x)/int psi on |x|<=1, zero outside (Eq. wfunc_pswf)."""
        x = np.asarray(x, dtype=np.float64)
        return np.where(np.abs(x) <= 1.0, npleg.legval(np.clip(x, -1, 1), self.phi_coef), 0.0)

    def dphi(self, x):
        x = np.asarray(x, dtype=np.float64)
        return np.where(np.abs(x) <= 1.0, npleg.legval(np.clip(x, -1, 1), self.dphi_coef), 0.0)

    def Phi(self, r):
        """Phi(r) = 1 - 2 int_0^r phi(t) dt for 0<=r<=1, 0 beyond (Eq. def_erfc_like_fcn)."""
        r = np.asarray(r, dtype=np.float64)
        val = 1.0 - 2.0 * npleg.legval(np.clip(r, 0.0, 1.0), self.iphi_coef)
        return np.where(r < 1.0, val, 0.0)

    # ---- Fourier-space window ---------------------------------------------
    def phihat(self, k):
        """phi-hat(k) = psi(k/c)/psi(0) for |k|<=c, zero beyond (Eq. wfunchat)."""
        k = np.asarray(k, dtype=np.float64)
        x = np.clip(k / self.c, -1.0, 1.0)
        return np.where(np.abs(k) <= self.c, npleg.legval(x, self.psi_coef) / self.psi0, 0.0)

    def dphihat(self, k):
        k = np.asarray(k, dtype=np.float64)
        x = np.clip(k / self.c, -1.0, 1.0)
        return np.where(np.abs(k) <= self.c,
                        npleg.legval(x, self.dpsi_coef) / (self.c * self.psi0), 0.0)

    def d2phihat0(self):
        """phi-hat''(0) (needed for the k -> 0 limit of the difference kernel)."""
        return npleg.legval(0.0, self.d2psi_coef) / (self.c * self.c * self.psi0)

    def gammaB_hat(self, k):
        """Biharmonic screening gammaB-hat(k) = phi-hat(k) - k phi-hat'(k)/2 (Eq. gammaB_in_phi)."""
        k = np.asarray(k, dtype=np.float64)
        return self.phihat(k) - 0.5 * k * self.dphihat(k)

    def phi0(self):
        return float(self.phi(0.0))
