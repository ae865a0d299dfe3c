"""Kernels, their residual parts and Fourier symbols (oracle; test infrastructure only).

Laplace: H = 1/(4 pi r), H_R = Phi(r/nu)/(4 pi r), H_M-hat = phi-hat(k nu)/k^2
(Eq. Hhatsplit_wfunc).  Stokes kernels (App. B, Eqs. stokeslet/stresslet/rotlet_def_deriv,
diffop-rel-fourier-S/T/R, res_stokeslet, res_stresslet, res_rotlet, Remark
scaling_stokes_split): the Stokeslet and stresslet come from the biharmonic kernel with
screening gammaB-hat, the rotlet from the harmonic kernel with screening phi-hat.

Layouts: strengths carry d_rho components (Laplace 1; Stokeslet force 3; stresslet
Q_lm = q_l n_m flattened l-major, 9; rotlet torque 3); potentials d_u components
(1, 3, 3, 3).  A kernel value is a (..., d_u, d_rho) array K with u_j = sum_a K_ja rho_a.

Every real-space function accepts complex displacements so that gradients can be
taken by complex-step differentiation (d f/dx = Im f(x + i h)/h).
"""
import numpy as np
from numpy.polynomial import legendre as npleg

from .params import D_RHO, D_U

EPS3 = np.zeros((3, 3, 3))
EPS3[0, 1, 2] = EPS3[1, 2, 0] = EPS3[2, 0, 1] = 1.0
EPS3[0, 2, 1] = EPS3[2, 1, 0] = EPS3[1, 0, 2] = -1.0
I3 = np.eye(3)


def _win_c(win, rho):
    """Phi, phi, phi' at (possibly complex) scaled radius rho < 1 (Eq. def_erfc_like_fcn)."""
    Phi = 1.0 - 2.0 * npleg.legval(rho, win.iphi_coef)
    phi = npleg.legval(rho, win.phi_coef)
    dphi = npleg.legval(rho, win.dphi_coef)
    return Phi, phi, dphi


class Kernel:
    def __init__(self, name):
        self.name = name
        self.d_rho = D_RHO[name]
        self.d_u = D_U[name]
        self.biharmonic = name in ("stokeslet", "stresslet")

    # ---- real space ----------------------------------------------------------
    def residual(self, dx, nu, win):
        """K_R(dx, nu) for displacements dx (n,3) with 0 < |dx| < nu; returns (n, d_u, d_rho).

        Laplace Eq. Hhatsplit_wfunc; Stokeslet Eqs. res_stokeslet/Soffdiag; stresslet
        Eqs. res_stresslet/T-offd; rotlet Eqs. res_rotlet/ROoffd, all at r/nu (Remark
        scaling_stokes_split).
        """
        r2 = np.sum(dx * dx, axis=1)
        r = np.sqrt(r2)
        rho = r / nu
        Phi, phi, dphi = _win_c(win, rho)
        n = dx.shape[0]
        if self.name == "laplace":
            return (Phi / (4 * np.pi * r)).reshape(n, 1, 1)
        if self.name == "stokeslet":
            Sd = Phi - 2 * rho * phi
            So = Phi + 2 * rho * phi
            xx = dx[:, :, None] * dx[:, None, :]
            return (Sd / (8 * np.pi * r))[:, None, None] * I3 + (So / (8 * np.pi * r ** 3))[:, None, None] * xx
        if self.name == "stresslet":
            Td = -2 * rho * rho * dphi
            To = Phi + 2 * rho * phi - (2.0 / 3.0) * rho * rho * dphi
            # T_jlm = (d_jl x_m + d_lm x_j + d_mj x_l)/(8 pi r^3) Td - 3/(4 pi) x_j x_l x_m / r^5 To
            t1 = (np.einsum("jl,nm->njlm", I3, dx) + np.einsum("lm,nj->njlm", I3, dx)
                  + np.einsum("mj,nl->njlm", I3, dx))
            t2 = np.einsum("nj,nl,nm->njlm", dx, dx, dx)
            T = (Td / (8 * np.pi * r ** 3))[:, None, None, None] * t1 \
                - (3.0 / (4 * np.pi) * To / r ** 5)[:, None, None, None] * t2
            return T.reshape(n, 3, 9)
        if self.name == "rotlet":
            Oo = Phi + 2 * rho * phi
            return (Oo / (8 * np.pi * r ** 3))[:, None, None] * np.einsum("jlm,nm->njl", EPS3, dx)
        raise ValueError(self.name)

    def full(self, dx):
        """The kernel itself, K(dx) (Sec. 1; App. B Eqs. stokeslet/stresslet/rotlet_def_deriv)."""
        r = np.sqrt(np.sum(dx * dx, axis=1))
        n = dx.shape[0]
        if self.name == "laplace":
            return (1 / (4 * np.pi * r)).reshape(n, 1, 1)
        if self.name == "stokeslet":
            xx = dx[:, :, None] * dx[:, None, :]
            return (1 / (8 * np.pi * r))[:, None, None] * I3 + (1 / (8 * np.pi * r ** 3))[:, None, None] * xx
        if self.name == "stresslet":
            t2 = np.einsum("nj,nl,nm->njlm", dx, dx, dx)
            return (-3.0 / (4 * np.pi) / r ** 5)[:, None, None] * t2.reshape(n, 3, 9)
        if self.name == "rotlet":
            return (1 / (8 * np.pi * r ** 3))[:, None, None] * np.einsum("jlm,nm->njl", EPS3, dx)
        raise ValueError(self.name)

    def self_matrix(self, nu, win):
        """lim_{r->0} K_M(r, nu) (Sec. 2.4; App. B Eq. S_self and Remark scaling_stokes_split)."""
        if self.name == "laplace":
            return np.full((1, 1), win.phi0() / (2 * np.pi * nu))
        if self.name == "stokeslet":
            return I3 * win.phi0() / (2 * np.pi * nu)
        return np.zeros((self.d_u, self.d_rho))

    def self_grad(self, nu, win):
        """g[i, j, a] = d_i K_M,ja(0, nu): the gradient part of the self correction (Sec. 2.4).

        Zero for the even kernels (Laplace, Stokeslet).  For the odd ones, expanding App. B's
        residual functions with phi(t) = phi(0) + phi''(0) t^2/2 + ...:
          rotlet    Omega_offd = 1 + (2/3) phi''(0) rho^3  =>  Omega_M,jl = -phi''(0) eps_jlm x_m/(12 pi nu^3)
          stresslet T_diag = -2 phi''(0) rho^3, T_offd = 1 + O(rho^5)
                    =>  T_M,jlm = phi''(0) (d_jl x_m + d_lm x_j + d_mj x_l)/(4 pi nu^3)
        """
        g = np.zeros((3, self.d_u, self.d_rho))
        d2 = float(npleg.legval(0.0, npleg.legder(win.phi_coef, 2)))
        if self.name == "rotlet":
            for i in range(3):
                g[i] = -d2 / (12 * np.pi * nu ** 3) * EPS3[:, :, i]
        elif self.name == "stresslet":
            T = np.zeros((3, 3, 3, 3))          # [i, j, l, m]
            for i in range(3):
                T[i] = (np.einsum("jl,m->jlm", I3, I3[i]) + np.einsum("lm,j->jlm", I3, I3[i])
                        + np.einsum("mj,l->jlm", I3, I3[i]))
            g = d2 / (4 * np.pi * nu ** 3) * T.reshape(3, 3, 9)
        return g

    # ---- Fourier space ---------------------------------------------------------
    def op_symbol(self, k):
        """Fourier symbol of the differential operator (Eqs. diffop-rel-fourier-S/T/R); (n,d_u,d_rho)."""
        n = k.shape[0]
        k2 = np.sum(k * k, axis=1)
        if self.name == "laplace":
            return np.ones((n, 1, 1), dtype=complex)
        if self.name == "stokeslet":
            return (k2[:, None, None] * I3 - k[:, :, None] * k[:, None, :]).astype(complex)
        if self.name == "stresslet":
            t1 = (np.einsum("nm,jl->njlm", k, I3) + np.einsum("nl,mj->njlm", k, I3)
                  + np.einsum("nj,lm->njlm", k, I3)) * k2[:, None, None, None]
            t2 = 2 * np.einsum("nj,nl,nm->njlm", k, k, k)
            return (1j * (t1 - t2)).reshape(n, 3, 9)
        if self.name == "rotlet":
            return -0.5j * np.einsum("jlm,nm->njl", EPS3, k)
        raise ValueError(self.name)

    def screening(self, kn, win):
        """gamma-hat: phi-hat (harmonic) or gammaB-hat (biharmonic), Sec. 5.1 and Eq. gammaB_in_phi."""
        return win.gammaB_hat(kn) if self.biharmonic else win.phihat(kn)

    def moll_symbol(self, k, nu, win):
        """K_M-hat(k, nu) = D-hat(k) gamma-hat(|k| nu)/|k|^{2 or 4} for k != 0 (App. B)."""
        kn = np.sqrt(np.sum(k * k, axis=1))
        pw = 4 if self.biharmonic else 2
        return self.op_symbol(k) * (self.screening(kn * nu, win) / kn ** pw)[:, None, None]

    def diff_symbol(self, k, nu_fine, nu_coarse, win):
        """D_l-hat(k) = K_M-hat(k, nu_{l+1}) - K_M-hat(k, nu_l) (Eq. diffkernel), with the k=0 limit.

        At k = 0: Laplace gives phi-hat''(0) (nu_f^2 - nu_c^2)/2 (Taylor expansion of the
        even phi-hat); the Stokes kernels give 0 because their operator symbol vanishes
        at k = 0 while the bracket stays bounded.
        """
        kn = np.sqrt(np.sum(k * k, axis=1))
        out = np.zeros((k.shape[0], self.d_u, self.d_rho), dtype=complex)
        nz = kn > 0
        if np.any(nz):
            pw = 4 if self.biharmonic else 2
            kk = k[nz]
            g = (self.screening(kn[nz] * nu_fine, win) - self.screening(kn[nz] * nu_coarse, win)) / kn[nz] ** pw
            out[nz] = self.op_symbol(kk) * g[:, None, None]
        if self.name == "laplace" and np.any(~nz):
            out[~nz] = win.d2phihat0() * (nu_fine ** 2 - nu_coarse ** 2) / 2
        return out


def get_kernel(name):
    return Kernel(name)
