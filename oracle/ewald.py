"""Independent reference sums for the Laplace kernel and the periodic Stokeslet (oracle; test
infrastructure only).

These do not use the DMK machinery, the PSWF window or truncated kernels: they
evaluate Eq. periodic_sum for K = 1/(4 pi r) through the classical Gaussian (Ewald)
split of Eq. ewald-split, H = erf(r/nu)/(4 pi r) + erfc(r/nu)/(4 pi r), with
H_M-hat = exp(-k^2 nu^2/4)/k^2 (Eq. Hhat_k):

  real space   sum over images within the erfc cutoff, excluding p = 0 when x_t = x_s;
  Fourier      D=3: Eq. ewald_far_3P_es with the Gaussian window (k = 0 dropped: neutral
               or neutralising background, Sec. 1 footnote);
               D=2: Eq. ewald_far_2P_es: for (k1,k2) != 0 the kappa_3 integral in closed
               form (checked against scipy quadrature in the tests); for (k1,k2) = 0 the
               neutral-regularised integral  int (e^{-k^2 nu^2/4} cos(kz) - 1)/k^2 dk
               up to its z-independent value at z = 0 (cancels for neutral charges);
               D=1: Eq. ewald_far_1P_es: the (kappa_2, kappa_3) integral in polar form,
               2 pi int_0^inf J0(kappa rho) e^{-(k1^2+kappa^2) nu^2/4}/(k1^2+kappa^2) kappa dkappa,
               by Gauss-Legendre quadrature for k1 != 0, and the neutral-regularised
               closed form for k1 = 0;
  self         - rho_t lim_{r->0} erf(r/nu)/(4 pi r) = - rho_t/(2 pi^{3/2} nu).
D = 0 is the plain O(N^2) sum.  Gradients (the field) are returned as well.

Stokeslet, D = 3, 2, 1: Hasimoto's split of the Oseen tensor (below), real-space images
within the cutoff plus the Fourier sum over k != 0 (D = 2: the kappa_3 integrals in closed
form; D = 1: the transverse integrals in polar form by Gauss-Legendre quadrature; the
non-periodic mode regularised for forces that sum to zero), minus the target's own smooth
part.
"""
import numpy as np
import scipy.special as sp

SQPI = np.sqrt(np.pi)


def direct_free(x, q, grad=False):
    """u_t = sum_{s != t} q_s/(4 pi |x_t - x_s|) (D = 0, Eq. periodic_sum)."""
    dx = x[:, None, :] - x[None, :, :]
    r = np.sqrt(np.sum(dx * dx, axis=2))
    np.fill_diagonal(r, np.inf)
    u = (q[None, :] / (4 * np.pi * r)).sum(axis=1)
    if not grad:
        return u
    g = -(dx * (q[None, :] / (4 * np.pi * r ** 3))[:, :, None]).sum(axis=1)
    return u, g


def _real_space(x, q, L, periodic, nu, grad):
    N = x.shape[0]
    rc = 6.5 * nu
    ranges = []
    for i in range(3):
        if periodic[i]:
            n = int(np.ceil(rc / L[i])) + 1
            ranges.append(np.arange(-n, n + 1))
        else:
            ranges.append(np.array([0]))
    u = np.zeros(N)
    g = np.zeros((N, 3))
    for a in ranges[0]:
        for b in ranges[1]:
            for c in ranges[2]:
                p = np.array([a * L[0], b * L[1], c * L[2]])
                dx = x[:, None, :] - x[None, :, :] + p
                r = np.sqrt(np.sum(dx * dx, axis=2))
                if a == 0 and b == 0 and c == 0:
                    np.fill_diagonal(r, np.inf)
                with np.errstate(divide="ignore", invalid="ignore"):
                    f = sp.erfc(r / nu) / (4 * np.pi * r)
                    f = np.where(np.isfinite(r), f, 0.0)
                u += (f * q[None, :]).sum(axis=1)
                if grad:
                    with np.errstate(divide="ignore", invalid="ignore"):
                        df = -(sp.erfc(r / nu) / r ** 2 + 2 / (SQPI * nu) * np.exp(-(r / nu) ** 2) / r) / (4 * np.pi)
                        df = np.where(np.isfinite(r), df / r, 0.0)
                    g += (dx * (df * q[None, :])[:, :, None]).sum(axis=1)
    return u, g


def _kmax(nu):
    # exp(-k^2 nu^2/4) < 1e-19
    return 2 * np.sqrt(44.0) / nu


def ewald_3p(x, q, L, nu, grad=False):
    u, g = _real_space(x, q, L, (True, True, True), nu, grad)
    km = _kmax(nu)
    n = [int(np.ceil(km * L[i] / (2 * np.pi))) for i in range(3)]
    ax = [2 * np.pi * np.arange(-n[i], n[i] + 1) / L[i] for i in range(3)]
    kk = np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)
    k2 = np.sum(kk * kk, axis=1)
    kk, k2 = kk[k2 > 0], k2[k2 > 0]
    w = np.exp(-k2 * nu * nu / 4) / k2 / (L[0] * L[1] * L[2])
    S = np.exp(-1j * x @ kk.T).T @ q              # sum_s q_s e^{-ik x_s}
    E = np.exp(1j * x @ kk.T)                     # (N, nk)
    u += (E @ (w * S)).real
    if grad:
        g += ((E * (1j * (w * S))[None, :]) @ kk).real
    u -= q / (2 * np.pi ** 1.5 * nu)
    return (u, g) if grad else u


def _int_2p(alpha, z, nu):
    """int e^{-(alpha^2+k^2) nu^2/4}/(alpha^2+k^2) e^{ikz} dk, alpha > 0 (closed form)."""
    e = np.exp(-alpha ** 2 * nu ** 2 / 4 - z ** 2 / nu ** 2)
    w1 = alpha * nu / 2 + z / nu
    w2 = alpha * nu / 2 - z / nu
    return np.pi / (2 * alpha) * e * (sp.erfcx(w1) + sp.erfcx(w2))


def _dint_2p(alpha, z, nu):
    """d/dz of _int_2p: the two Gaussian terms from differentiating erfc cancel, leaving
    (pi/2) (e^{az} erfc(a nu/2 + z/nu) - e^{-az} erfc(a nu/2 - z/nu))."""
    e = np.exp(-alpha ** 2 * nu ** 2 / 4 - z ** 2 / nu ** 2)
    w1 = alpha * nu / 2 + z / nu
    w2 = alpha * nu / 2 - z / nu
    return np.pi / 2 * e * (sp.erfcx(w1) - sp.erfcx(w2))


def ewald_2p(x, q, L, nu, grad=False):
    u, g = _real_space(x, q, L, (True, True, False), nu, grad)
    km = _kmax(nu)
    n = [int(np.ceil(km * L[i] / (2 * np.pi))) for i in range(2)]
    A = 1.0 / (L[0] * L[1] * 2 * np.pi)
    dz = x[:, None, 2] - x[None, :, 2]
    for a in range(-n[0], n[0] + 1):
        for b in range(-n[1], n[1] + 1):
            k1, k2 = 2 * np.pi * a / L[0], 2 * np.pi * b / L[1]
            if a == 0 and b == 0:
                # int (e^{-k^2nu^2/4} cos kz - 1)/k^2 dk = -pi (z erf(z/nu) + nu/sqrt(pi)(e^{-z^2/nu^2} - 1))
                I0 = -np.pi * (dz * sp.erf(dz / nu) + nu / SQPI * (np.exp(-(dz / nu) ** 2) - 1))
                u += A * (I0 * q[None, :]).sum(axis=1)
                if grad:
                    dI0 = -np.pi * sp.erf(dz / nu)
                    g[:, 2] += A * (dI0 * q[None, :]).sum(axis=1)
                continue
            al = np.hypot(k1, k2)
            if al * nu / 2 > np.sqrt(44.0):
                continue
            I = _int_2p(al, dz, nu)
            ph = np.exp(1j * (k1 * (x[:, None, 0] - x[None, :, 0]) + k2 * (x[:, None, 1] - x[None, :, 1])))
            u += A * (ph * I * q[None, :]).sum(axis=1).real
            if grad:
                g[:, 0] += A * (1j * k1 * ph * I * q[None, :]).sum(axis=1).real
                g[:, 1] += A * (1j * k2 * ph * I * q[None, :]).sum(axis=1).real
                g[:, 2] += A * (ph * _dint_2p(al, dz, nu) * q[None, :]).sum(axis=1).real
    u -= q / (2 * np.pi ** 1.5 * nu)
    return (u, g) if grad else u


def _polar_1p(k1, rr, nu, nq=600):
    """2 pi int_0^inf J0(kappa rho) e^{-(k1^2+kappa^2)nu^2/4}/(k1^2+kappa^2) kappa dkappa and d/drho."""
    kmx = _kmax(nu)
    t, wt = np.polynomial.legendre.leggauss(nq)
    kap = 0.5 * kmx * (t + 1)
    wt = 0.5 * kmx * wt
    f = np.exp(-(k1 ** 2 + kap ** 2) * nu ** 2 / 4) / (k1 ** 2 + kap ** 2) * kap * wt
    J0 = sp.j0(np.multiply.outer(rr, kap))
    J1 = sp.j1(np.multiply.outer(rr, kap))
    val = 2 * np.pi * (J0 @ f)
    dval = 2 * np.pi * ((-J1 * kap) @ f)
    return val, dval


def ewald_1p(x, q, L, nu, grad=False):
    u, g = _real_space(x, q, L, (True, False, False), nu, grad)
    km = _kmax(nu)
    n = int(np.ceil(km * L[0] / (2 * np.pi)))
    A = 1.0 / (L[0] * (2 * np.pi) ** 2)
    dy = x[:, None, 1] - x[None, :, 1]
    dzz = x[:, None, 2] - x[None, :, 2]
    rr = np.sqrt(dy ** 2 + dzz ** 2)
    dx1 = x[:, None, 0] - x[None, :, 0]
    for a in range(-n, n + 1):
        k1 = 2 * np.pi * a / L[0]
        if a == 0:
            # 2 pi int_0^inf (J0(kappa rho) - 1) e^{-kappa^2 nu^2/4}/kappa dkappa
            #   = -pi (E1(rho^2/nu^2) + ln(rho^2/nu^2) + gamma)
            with np.errstate(divide="ignore", invalid="ignore"):
                xx = (rr / nu) ** 2
                I0 = -np.pi * (sp.exp1(xx) + np.log(xx) + np.euler_gamma)
                I0 = np.where(rr > 0, I0, 0.0)
            u += A * (I0 * q[None, :]).sum(axis=1)
            if grad:
                with np.errstate(divide="ignore", invalid="ignore"):
                    dI0 = -2 * np.pi * (1 - np.exp(-(rr / nu) ** 2)) / rr
                    dI0 = np.where(rr > 0, dI0, 0.0)
                    cy = np.where(rr > 0, dy / rr, 0.0)
                    cz = np.where(rr > 0, dzz / rr, 0.0)
                g[:, 1] += A * (dI0 * cy * q[None, :]).sum(axis=1)
                g[:, 2] += A * (dI0 * cz * q[None, :]).sum(axis=1)
            continue
        if abs(k1) * nu / 2 > np.sqrt(44.0):
            continue
        I, dI = _polar_1p(k1, rr, nu)
        ph = np.exp(1j * k1 * dx1)
        u += A * (ph * I * q[None, :]).sum(axis=1).real
        if grad:
            with np.errstate(divide="ignore", invalid="ignore"):
                cy = np.where(rr > 0, dy / rr, 0.0)
                cz = np.where(rr > 0, dzz / rr, 0.0)
            g[:, 0] += A * (1j * k1 * ph * I * q[None, :]).sum(axis=1).real
            g[:, 1] += A * (ph * dI * cy * q[None, :]).sum(axis=1).real
            g[:, 2] += A * (ph * dI * cz * q[None, :]).sum(axis=1).real
    u -= q / (2 * np.pi ** 1.5 * nu)
    return (u, g) if grad else u


def laplace_reference(D, L, x, q, nu=None, grad=False):
    """Reference u (and field gradient) for the Laplace kernel with D periodic directions."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64).ravel()
    if D == 0:
        return direct_free(x, q, grad)
    if nu is None:
        nu = min(L[:D]) / 4
    return {3: ewald_3p, 2: ewald_2p, 1: ewald_1p}[D](x, q, list(L), nu, grad)


# ---- Stokeslet, triply periodic: Hasimoto's split of the Oseen tensor ----------------------
#
# G(x) = (delta/r + x x^T/r^3)/(8 pi), G-hat(k) = (I - k k^T/k^2)/k^2 (unit viscosity), split as
# G-hat = G-hat (1 - phi) + G-hat phi with phi(k) = (1 + k^2 nu^2/4) e^{-k^2 nu^2/4} (Hasimoto,
# J. Fluid Mech. 5 (1959)).  The smooth part in real space, written with the Laplace Gaussian
# split H_M = erf(r/nu)/(4 pi r) (H_M-hat = e^{-k^2 nu^2/4}/k^2), the Gaussian
# g = e^{-r^2/nu^2}/(pi^{3/2} nu^3) (g-hat = e^{-k^2 nu^2/4}) and the radial V with
# laplacian(V) = H_M (V-hat = -e^{-k^2 nu^2/4}/k^4):
#
#   G^F = I (H_M + nu^2/4 g) - grad grad V + nu^2/4 grad grad H_M,
#   r^2 V'(r) = [(r^2/2 - nu^2/4) erf(r/nu) + nu r/(2 sqrt(pi)) e^{-r^2/nu^2}]/(4 pi),
#
# and G^R = G - G^F decays like e^{-r^2/nu^2}.  grad grad f = f'' xx^T/r^2 + f'/r (I - xx^T/r^2)
# for radial f.  G^F(0) = I/(2 pi^{3/2} nu) (the smooth self term).  The tests check G^F against
# the inverse Fourier transform of G-hat phi by radial quadrature.

def _stokes_smooth_radial(r, nu):
    """(a, b) with G^F(x) = a(r) I + b(r) x x^T/r^2 (r > 0; complex r allowed)."""
    E = sp.erf(r / nu)
    e = np.exp(-(r / nu) ** 2)
    H = E / (4 * np.pi * r)
    Hp = (2 * r / (SQPI * nu) * e - E) / (4 * np.pi * r ** 2)
    Hpp = (-4 * e / (SQPI * nu ** 3) - 4 * e / (SQPI * nu * r ** 2) + 2 * E / r ** 3) / (4 * np.pi)
    g = e / (np.pi ** 1.5 * nu ** 3)
    Nr = (r * r / 2 - nu * nu / 4) * E + nu * r / (2 * SQPI) * e
    Vp = Nr / (4 * np.pi * r ** 2)
    Vpp = (r * r * E - 2 * Nr) / (4 * np.pi * r ** 3)
    q = nu * nu / 4
    # I part: H + q g - V'/r + q H'/r ; xx part: -(V'' - V'/r) + q (H'' - H'/r)
    a = H + q * g - Vp / r + q * Hp / r
    b = -(Vpp - Vp / r) + q * (Hpp - Hp / r)
    return a, b


def stokes_smooth(x, nu):
    """G^F at displacements x (n, 3), r > 0: (n, 3, 3)."""
    r = np.sqrt(np.sum(x * x, axis=-1))
    a, b = _stokes_smooth_radial(r, nu)
    xx = x[:, :, None] * x[:, None, :] / (r * r)[:, None, None]
    return a[:, None, None] * np.eye(3) + b[:, None, None] * xx


def _stokes_real(xt, xs, f, L, periodic, nu):
    """Real-space part: sum over the images within the cutoff of G^R(x_t - x_s + p) f_s."""
    N = xs.shape[0]
    rc = 6.5 * nu
    n = [int(np.ceil(rc / L[i])) + 1 if periodic[i] else 0 for i in range(3)]
    u = np.zeros((xt.shape[0], 3), dtype=np.result_type(xt, 1.0))
    same = np.eye(xt.shape[0], N, dtype=bool)
    for a in range(-n[0], n[0] + 1):
        for b in range(-n[1], n[1] + 1):
            for c in range(-n[2], n[2] + 1):
                p = np.array([a * L[0], b * L[1], c * L[2]])
                dx = xt[:, None, :] - xs[None, :, :] + p
                keep = ~same if (a == 0 and b == 0 and c == 0) else np.ones_like(same)
                d = dx[keep]
                r = np.sqrt(np.sum(d * d, axis=-1))
                aa, bb = _stokes_smooth_radial(r, nu)
                # G^R = G - G^F = (1/(8 pi r) - a) I + (1/(8 pi r) - b) x x^T/r^2
                ci = 1 / (8 * np.pi * r) - aa
                cx = 1 / (8 * np.pi * r) - bb
                fs = np.broadcast_to(f[None, :, :], dx.shape)[keep]
                v = ci[:, None] * fs + (cx * np.sum(d * fs, axis=-1) / (r * r))[:, None] * d
                tt = np.nonzero(keep)[0]
                np.add.at(u, tt, v)
    return u


def stokeslet_ewald_3p(xt, xs, f, L, nu):
    """Velocities u_t = sum_s sum*_p G(x_t - x_s + p) f_s for D = 3 (k = 0 excluded), at the
    targets xt (n, 3; may be complex for complex-step derivatives) from sources xs (N, 3)
    with forces f (N, 3); target t and source t are the same point (p = 0 skipped)."""
    u = _stokes_real(xt, xs, f, L, (True, True, True), nu)
    # Fourier part, real form (analytic in xt)
    km = _kmax(nu)
    m = [int(np.ceil(km * L[i] / (2 * np.pi))) for i in range(3)]
    ax = [2 * np.pi * np.arange(-m[i], m[i] + 1) / L[i] for i in range(3)]
    kk = np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)
    k2 = np.sum(kk * kk, axis=1)
    kk, k2 = kk[k2 > 0], k2[k2 > 0]
    phi = (1 + k2 * nu * nu / 4) * np.exp(-k2 * nu * nu / 4) / k2 / (L[0] * L[1] * L[2])
    ks = xs @ kk.T                                     # (N, nk)
    C = np.cos(ks).T @ f                               # (nk, 3) sum_s f_s cos(k x_s)
    S = np.sin(ks).T @ f
    kt = xt @ kk.T                                     # (n, nk)
    for A, trig in ((C, np.cos(kt)), (S, np.sin(kt))):
        Ap = A - kk * (np.sum(kk * A, axis=1) / k2)[:, None]     # (I - k k^T/k^2) A
        u = u + trig @ (phi[:, None] * Ap)
    # the target's own smooth part
    u = u - f[: xt.shape[0]] / (2 * np.pi ** 1.5 * nu)
    return u


# ---- Stokeslet, doubly periodic (D = 2, x3 free) -----------------------------------------
#
# Same split; the Fourier part integrates G-hat phi over kappa_3 in closed form.  With
# I_L(alpha, z) = int e^{-(alpha^2+k^2) nu^2/4}/(alpha^2+k^2) e^{ikz} dk (_int_2p) and
# k^2 = alpha^2 + kappa_3^2, k = (k1, k2, kappa_3):
#   I0 = int phi/k^2 e^{ikz}  = I_L + (sqrt(pi) nu/2) e^{-alpha^2 nu^2/4 - z^2/nu^2},
#   I2 = int phi/k^4 e^{ikz}  = -d I_L/d(alpha^2),
#   dI2/dz                    = -(z/2) I_L.
# Per in-plane mode (k1, k2) != 0, M = int (I - k k^T/k^2) phi/k^2 e^{ikz} dk has the entries
#   M_ab = I0 delta_ab - k_a k_b I2 (a, b in-plane),  M_a3 = M_3a = -k_a int kappa_3 phi/k^4 e^{ikz}
#        = i k_a dI2/dz = -i k_a (z/2) I_L,  M_33 = I0 - (I0 - alpha^2 I2) = alpha^2 I2.
# The mode (0, 0) projects out x3 and leaves, for in-plane forces that sum to zero,
#   M_aa = int (e^{-k^2 nu^2/4} cos kz - 1)/k^2 dk + (sqrt(pi) nu/2) e^{-z^2/nu^2}.

def _stokes_2p_modes(alpha, z, nu):
    """(I0, I2, I_L) of the comment above, alpha > 0 (arrays; complex z allowed)."""
    IL = _int_2p(alpha, z, nu)
    E = np.exp(-alpha ** 2 * nu ** 2 / 4 - z ** 2 / nu ** 2)
    w1 = alpha * nu / 2 + z / nu
    w2 = alpha * nu / 2 - z / nu
    dIL = -IL / alpha + np.pi / (2 * alpha) * E * (z * (sp.erfcx(w1) - sp.erfcx(w2)) - 2 * nu / SQPI)
    I0 = IL + SQPI * nu / 2 * E
    I2 = -dIL / (2 * alpha)
    return I0, I2, IL


def stokeslet_ewald_2p(xt, xs, f, L, nu):
    """As stokeslet_ewald_3p for D = 2 (x1, x2 periodic, x3 free); the in-plane force
    components must sum to zero (the (0, 0) mode drops their divergent constant)."""
    u = _stokes_real(xt, xs, f, L, (True, True, False), nu)
    km = _kmax(nu)
    n = [int(np.ceil(km * L[i] / (2 * np.pi))) for i in range(2)]
    A = 1.0 / (L[0] * L[1] * 2 * np.pi)
    dx = xt[:, None, :] - xs[None, :, :]
    z = dx[:, :, 2]
    for a in range(-n[0], n[0] + 1):
        for b in range(-n[1], n[1] + 1):
            k1, k2 = 2 * np.pi * a / L[0], 2 * np.pi * b / L[1]
            if a == 0 and b == 0:
                I00 = -np.pi * (z * sp.erf(z / nu) + nu / SQPI * (np.exp(-(z / nu) ** 2) - 1))
                w = A * (I00 + SQPI * nu / 2 * np.exp(-(z / nu) ** 2))
                u[:, 0] = u[:, 0] + w @ f[:, 0]
                u[:, 1] = u[:, 1] + w @ f[:, 1]
                continue
            al = np.hypot(k1, k2)
            if al * nu / 2 > np.sqrt(44.0):
                continue
            I0, I2, IL = _stokes_2p_modes(al, z, nu)
            th = k1 * dx[:, :, 0] + k2 * dx[:, :, 1]
            c, sn = np.cos(th), np.sin(th)
            kv = (k1, k2)
            # real part of M e^{i th}: real entries times cos(th); the (a, 3) entries
            # -i k_a (z/2) I_L give +k_a (z/2) I_L sin(th)
            for j in range(3):
                for l in range(3):
                    if j < 2 and l < 2:
                        term = ((I0 if j == l else 0.0) - kv[j] * kv[l] * I2) * c
                    elif j == 2 and l == 2:
                        term = (al * al * I2) * c
                    else:
                        ka = kv[j] if j < 2 else kv[l]
                        term = ka * z / 2 * IL * sn
                    u[:, j] = u[:, j] + A * (term @ f[:, l])
    u = u - f[: xt.shape[0]] / (2 * np.pi ** 1.5 * nu)
    return u


# ---- Stokeslet, singly periodic (D = 1, x1 periodic) -------------------------------------
#
# Same split; the transverse wavevector q = (kappa_2, kappa_3), |q| = kappa, is integrated in
# polar form about rho = (x2, x3) differences, r = |rho|, with the angular means
#   <e^{iq.rho}> = J0(kappa r),  <q_a e^{iq.rho}> = i kappa J1(kappa r) rhohat_a,
#   <q_a q_b e^{iq.rho}> = kappa^2/2 [(J0 + J2) delta_ab - 2 J2 rhohat_a rhohat_b].
# With h0 = phi/k^2, h2 = phi/k^4 (k^2 = k1^2 + kappa^2) and the radial integrals (Gauss-Legendre
# on [0, kmax]) P0 = 2 pi int h0 J0 kappa, Q0 = 2 pi int h2 J0 kappa, P1 = 2 pi int h2 J1 kappa^2,
# R0 = pi int h2 (J0 + J2) kappa^3, R2 = 2 pi int h2 J2 kappa^3, a mode k1 != 0 contributes
#   M_11 = P0 - k1^2 Q0,  M_1a = M_a1 = -i k1 P1 rhohat_a,  M_ab = (P0 - R0) delta_ab + R2 rhohat rhohat.
# The mode k1 = 0 (q only) keeps, for forces that sum to zero, M_11 = the Laplace regularised
# integral -pi (E1(r^2/nu^2) + ln(r^2/nu^2) + gamma) + pi e^{-r^2/nu^2} and
#   M_ab = pi int [phi (J0 - J2) - e^{-kappa^2 nu^2/4}]/kappa delta_ab + 2 pi int phi J2/kappa rhohat rhohat.

def stokeslet_ewald_1p(xt, xs, f, L, nu, nq=800):
    """As stokeslet_ewald_3p for D = 1 (x1 periodic; x2, x3 free); the force components must
    sum to zero (the k1 = 0 mode drops their divergent constant)."""
    u = _stokes_real(xt, xs, f, L, (True, False, False), nu)
    km = _kmax(nu)
    t, wt = np.polynomial.legendre.leggauss(nq)
    kap = 0.5 * km * (t + 1)
    wt = 0.5 * km * wt
    dx = xt[:, None, :] - xs[None, :, :]
    # a target's own term is even in the displacement: taken at displacement 0 (constant in xt)
    same = np.eye(xt.shape[0], xs.shape[0], dtype=bool)
    dx = np.where(same[..., None], 0.0, dx)
    r = np.sqrt(dx[:, :, 1] ** 2 + dx[:, :, 2] ** 2)
    zero = same
    rz = np.where(zero, 1.0, r)
    rh = [np.where(zero, 0.0, dx[:, :, 1 + i] / rz) for i in range(2)]
    kr = r[:, :, None] * kap
    J0, J1, J2 = sp.jv(0, kr), sp.jv(1, kr), sp.jv(2, kr)
    n = int(np.ceil(km * L[0] / (2 * np.pi)))
    A = 1.0 / (L[0] * (2 * np.pi) ** 2)
    for a in range(-n, n + 1):
        k1 = 2 * np.pi * a / L[0]
        if a == 0:
            e = np.exp(-kap ** 2 * nu ** 2 / 4)
            phi = (1 + kap ** 2 * nu ** 2 / 4) * e
            xx = np.where(zero, 1.0, r * r / (nu * nu))
            m11 = -np.pi * (sp.exp1(xx) + np.log(xx) + np.euler_gamma) + np.pi * np.exp(-xx)
            M11 = np.where(zero, np.pi, m11)           # its limit at r = 0
            T0 = np.pi * (((phi * (J0 - J2) - e) / kap) @ wt)
            T2 = 2 * np.pi * ((phi * J2 / kap) @ wt)
            C1 = 0.0 * M11
        else:
            if abs(k1) * nu / 2 > np.sqrt(44.0):
                continue
            k2 = k1 * k1 + kap ** 2
            phi = (1 + k2 * nu * nu / 4) * np.exp(-k2 * nu * nu / 4)
            h0, h2 = phi / k2 * wt, phi / k2 ** 2 * wt
            P0 = 2 * np.pi * (J0 @ (h0 * kap))
            M11 = P0 - k1 * k1 * 2 * np.pi * (J0 @ (h2 * kap))
            C1 = k1 * 2 * np.pi * (J1 @ (h2 * kap ** 2))      # M_1a = -i C1 rhohat_a
            T0 = P0 - np.pi * ((J0 + J2) @ (h2 * kap ** 3))
            T2 = 2 * np.pi * (J2 @ (h2 * kap ** 3))
        # real part of M e^{i k1 d1}: the real entries times cos; -i C1 rhohat_a gives
        # +C1 rhohat_a sin (written without real parts, so that it is analytic in xt)
        c, sn = np.cos(k1 * dx[:, :, 0]), np.sin(k1 * dx[:, :, 0])
        u[:, 0] = u[:, 0] + A * ((M11 * c) @ f[:, 0])
        for i in range(2):
            cross = C1 * rh[i] * sn
            u[:, 0] = u[:, 0] + A * (cross @ f[:, 1 + i])
            u[:, 1 + i] = u[:, 1 + i] + A * (cross @ f[:, 0])
            for j in range(2):
                Mij = (T0 if i == j else 0.0) + T2 * rh[i] * rh[j]
                u[:, 1 + i] = u[:, 1 + i] + A * ((Mij * c) @ f[:, 1 + j])
    u = u - f[: xt.shape[0]] / (2 * np.pi ** 1.5 * nu)
    return u
