"""Plan parameters (oracle; test infrastructure only).

Sec. 6.1 and Tables 1 (Laplace) and 5 (Stokes kernels) fix, per tolerance row,
the PSWF band limit c and the Chebyshev order p.  Readings taken here:

* tol in between rows maps to the next stricter row (1e-3, 1e-6, 1e-9, 1e-12).
* c is taken as printed in Tables 1 and 5, with one exception: the rotlet
  1e-3 row prints 6.28, and only c = 2 pi (which 6.28 rounds) reproduces its
  N_per = 3; with the printed values every other N_F and N_per of both tables
  follows from the rules below.
* n_f = ceil(3c/pi) - 1 and N_F = 2 n_f + 1 (Sec. 6.1; the text of Sec. 2.3
  omits the -1, the tables use it).  The ceiling is taken after removing a
  relative 1e-12 so that 3c/pi landing on an integer does not round up.
* nu_0 = s, the root cube side (Sec. 4: supp D_l = r_l = box side, and Table 1
  gives R = L_3 + nu_0 = 2 on the unit cube).
* Root modes: the periodic integer range of Eq. kintmax (ceil), keeping only
  |k| nu_0 <= c (phi-hat is zero beyond the band, Eq. wfunchat), with ties kept
  up to a relative 1e-12.  This reproduces every N_per of Tables 1 and 5 except
  where c/(2 pi) is itself an integer (a tie whose mode carries phi-hat(c)).
* Free directions (Sec. 5.3, Eq. k1set-1p, k1k2set-2p): step dk = pi/R (the
  Nyquist limit for a kernel truncated at R, Sec. 5.3), n = -N..N with N the count of Eq.
  k1k2set-2p, (N-1) dk <= c/nu_0 <= N dk; where c/(nu_0 dk) is an integer (to a relative
  1e-12) both N = c/(nu_0 dk) and N + 1 satisfy it, and the larger is taken (it reproduces the
  rotlet rows of Table 5 at 1e-3, c = 2 pi); otherwise N = ceil(c/(nu_0 dk)); R = L_3 + nu_0 (D=2), sqrt((L_2+nu_0)^2+(L_3+nu_0)^2) (D=1), with
  the free lengths rounded up to multiples of s (Sec. 5).
* Original vs truncated symbol for the nonzero periodic modes (D = 1, 2; Sec. 5.3, App. E):
  the trapezoidal-rule error estimates of App. E (m = 1 for the harmonic kernels, Laplace and
  rotlet; m = 2 with C_gamma = 0 for the biharmonic ones, Stokeslet and stresslet) at
  alpha = alpha_min, |b| = L_j (the free extent of Omega_ext) and the Nyquist step of the
  original kernel h_j = pi/L_j, for each free direction.  If every one is at most tol (D = 1:
  Eq. app_1P_error_estimate sums the two; the sum would exceed 1e-3 on the unit cell for the
  harmonic kernels, 1.9e-3, and keep the truncated symbol there, whereas the D = 1 free counts
  of Tables 1 and 5 at 1e-3 are those of the original symbol's step -- the per-direction test
  reproduces them), the original symbol on the step-pi/L_j grid serves every mode with
  alpha != 0 and the truncated symbol on the step-pi/R grid the alpha = 0 modes (Eq.
  ewald_far_es_1P_discr_b and its D = 2 analogue); otherwise the truncated symbol serves every
  mode (Remark alpha_switch).
* D = 0: one cube of side max L_i (Sec. 3.1.1 "box of equal sides"); the root
  far field is the free-space Fourier integral of the kernel truncated at
  R = sqrt(sum (L_i+nu_0)^2) (Sec. 3.1.3), on the same trapezoidal grid rule.
"""
import math
import numpy as np

KERNELS = ("laplace", "stokeslet", "stresslet", "rotlet")
TOL_ROWS = (1e-3, 1e-6, 1e-9, 1e-12)

# (c, p) per tolerance row: Table 1 (Laplace) and Table 5 (Stokes kernels).
TABLE = {
    "laplace":   [(7.00, 12), (14.50, 20), (21.50, 30), (29.00, 38)],
    "stokeslet": [(10.47, 13), (17.80, 23), (25.13, 34), (32.46, 44)],
    "stresslet": [(10.47, 12), (17.80, 23), (25.13, 33), (33.51, 45)],
    "rotlet":    [(2 * math.pi, 8), (13.61, 18), (20.94, 29), (28.27, 39)],
}

# source/target component counts (App. B): Laplace scalar; Stokeslet force -> velocity;
# stresslet Q_lm = q_l n_m (9) -> velocity; rotlet torque -> velocity.
D_RHO = {"laplace": 1, "stokeslet": 3, "stresslet": 9, "rotlet": 3}
D_U = {"laplace": 1, "stokeslet": 3, "stresslet": 3, "rotlet": 3}


def table_row(tol):
    """Index of the tolerance row used for tol (next stricter row)."""
    if not (1e-12 * (1 - 1e-9) <= tol <= 1e-3 * (1 + 1e-9)):
        raise ValueError("tol outside [1e-12, 1e-3]")
    for i, t in enumerate(TOL_ROWS):
        if tol >= t * (1 - 1e-9):
            return i
    return len(TOL_ROWS) - 1


def c_and_p(kernel, tol):
    return TABLE[kernel][table_row(tol)]


def n_f(c):
    """n_f = ceil(3c/pi) - 1 (Sec. 6.1)."""
    return int(math.ceil(3.0 * c / math.pi * (1.0 - 1e-12))) - 1


class Geometry:
    """Cube tiling of the primary cell (Sec. 4.1.1-4.1.3, Sec. 5).

    Cubes of side s = the shortest periodic length (the largest length for D = 0).  A periodic
    direction whose length is an integer multiple of s is tiled exactly and stays periodic in
    the forest.  Any other periodic direction i (Sec. 4.1.1, non-exact tiling) is covered by
    ceil(L_i/s) cubes, the last of them cut, plus one padding cube on each side:
    Omega_ext spans [-s, s (ceil(L_i/s) + 1)) along i, the forest is non-periodic along i, and
    the periodic images of the sources that fall in Omega_ext are added as extra sources
    (Sec. 4.1.2).  Free directions: lengths rounded up to multiples of s (Sec. 5).

    Attributes: L (true lengths), s, M (cubes per axis, padding included), origin (lower
    corner of Omega_ext), Lext (extent of the cube tiling per axis), periodic (the sum is
    periodic along the axis), fperiodic (the forest wraps along the axis), padded.
    """

    def __init__(self, D, L):
        L = [float(v) for v in L]
        if D not in (0, 1, 2, 3):
            raise ValueError("D must be 0..3")
        if any(not (v > 0 and math.isfinite(v)) for v in L):
            raise ValueError("lengths must be positive")
        self.D = D
        self.L = L
        self.s = min(L[:D]) if D > 0 else max(L)
        M, Lext, origin, fper, pad = [], [], [], [], []
        for i in range(3):
            ratio = L[i] / self.s
            if i < D:
                m = int(round(ratio))
                if abs(ratio - m) <= 1e-12 * max(1.0, ratio):      # exact tiling
                    M.append(m)
                    Lext.append(L[i])
                    origin.append(0.0)
                    fper.append(True)
                    pad.append(False)
                else:                                               # cut cubes + padding
                    m = int(math.ceil(ratio * (1 - 1e-12))) + 2
                    M.append(m)
                    Lext.append(m * self.s)
                    origin.append(-self.s)
                    fper.append(False)
                    pad.append(True)
            else:
                m = int(math.ceil(ratio * (1 - 1e-12)))
                M.append(max(m, 1))
                Lext.append(M[-1] * self.s)
                origin.append(0.0)
                fper.append(False)
                pad.append(False)
        self.M = tuple(M)
        self.Lext = Lext
        self.origin = tuple(origin)
        self.nu0 = self.s
        self.periodic = tuple(i < D for i in range(3))
        self.fperiodic = tuple(fper)
        self.padded = tuple(pad)


def root_modes(kernel, geom, c, return_axes=False):
    """Root Fourier discretisation: list of wave vectors and the constant C^{DP}.

    Returns (k (n,3), C, R, dk); with return_axes, the three 1-D wavenumber axes of the
    enclosing rectangle and the boolean mask of retained modes on it instead of k.  Sec. 4.3 (Eq. wavenumbers-3p-trunc, kintmax) for the
    periodic directions and Sec. 5.3 (Eqs. k1set-1p, k1k2set-2p, ewald_far_allP_discr)
    for the free ones; D=0 by the same rule in all three directions.
    """
    D, nu0 = geom.D, geom.nu0
    K = c / nu0
    axes = []
    R = None
    dk = None
    Lx = geom.Lext
    if D == 3:
        pass
    elif D == 2:
        R = Lx[2] + nu0
    elif D == 1:
        R = math.sqrt((Lx[1] + nu0) ** 2 + (Lx[2] + nu0) ** 2)
    else:
        R = math.sqrt(sum((Lx[i] + nu0) ** 2 for i in range(3)))
    if D < 3:
        dk = math.pi / R
        Nfree = free_count(K, dk)
    for i in range(3):
        if i < D:
            kmax = int(math.ceil(geom.L[i] * K / (2 * math.pi) * (1 - 1e-12)))
            axes.append(2 * math.pi * np.arange(-kmax, kmax + 1) / geom.L[i])
        else:
            axes.append(dk * np.arange(-Nfree, Nfree + 1))
    kk = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    kn = np.sqrt(np.sum(kk * kk, axis=1))
    keep = kn * nu0 <= c * (1 + 1e-12)
    if D == 3:
        keep &= kn > 0
    keepr = keep.reshape(len(axes[0]), len(axes[1]), len(axes[2]))
    kk = kk[keep]
    if D == 3:
        C = 1.0 / (geom.L[0] * geom.L[1] * geom.L[2])
    elif D == 2:
        C = dk / (geom.L[0] * geom.L[1] * 2 * math.pi)
    elif D == 1:
        C = dk * dk / (geom.L[0] * (2 * math.pi) ** 2)
    else:
        C = dk ** 3 / (2 * math.pi) ** 3
    if return_axes:
        return axes, keepr, C, R, dk
    return kk, C, R, dk


def free_count(K, h):
    """N of the free set n = -N..N (Eqs. k1set-1p, k1k2set-2p): the smallest N with N h > K,
    i.e. ceil(K/h), plus one where K/h is an integer to a relative 1e-12."""
    return int(math.floor(K / h * (1 + 1e-12))) + 1


def mode_counts(kernel, D, L, tol):
    """(N_per_i, N_free_i, R) in the layout of Tables 1 and 5 (Sec. 6.1); N_free_i counts the
    nodes of the alpha != 0 modes (those of the original symbol's step pi/L_j where the App. E
    switch chooses it)."""
    c, p = c_and_p(kernel, tol)
    g = Geometry(D, L)
    kk, C, R, dk = root_modes(kernel, g, c)
    orig = original_symbol_ok(kernel, g, tol)
    counts = []
    for i in range(3):
        if i < D:       # N_per_i = number of distinct periodic integers kept
            vals = np.unique(np.round(kk[:, i] / (2 * math.pi / g.L[i])).astype(int))
            counts.append(len(vals))
        else:           # N_free_i = 2N+1 trapezoidal nodes of Eq. k1set-1p / k1k2set-2p
            h = math.pi / g.Lext[i] if orig else dk
            counts.append(2 * free_count(c / g.nu0, h) + 1)
    return counts, R


def free_error_estimate(m, alpha, s, h, C_gamma=0.0):
    """App. E (Eqs. app_m1_error_estimate, app_m2_error_estimate): the error of the infinite
    trapezoidal rule with step h for the model integral I_m(alpha, b), |b| = s, from the poles
    at kappa = +-i alpha.  With x = 2 pi alpha / h and E = e^x - 1, cosh(alpha s)/E and
    sinh(alpha s)/E are formed as exponentials of differences (no overflow for large x)."""
    x = 2 * math.pi * alpha / h
    den = -math.expm1(-x)                                  # E e^{-x}
    ch = 0.5 * (math.exp(alpha * s - x) + math.exp(-alpha * s - x)) / den      # cosh(alpha s)/E
    if m == 1:
        return 2 * math.pi / alpha * ch
    sh = 0.5 * (math.exp(alpha * s - x) - math.exp(-alpha * s - x)) / den      # sinh(alpha s)/E
    Einv = math.exp(-x) / den                                                  # 1/E
    return math.pi / alpha ** 3 * abs(ch - alpha * (s - alpha * C_gamma) * sh + x * ch * (1 + Einv))


def original_symbol_ok(kernel, geom, tol):
    """The App. E switch (Sec. 5.3): True if the original symbol may serve the alpha != 0 modes."""
    D = geom.D
    if D not in (1, 2):
        return False
    L = geom.L
    alpha = 2 * math.pi / (max(L[0], L[1]) if D == 2 else L[0])      # Eq. alphamin
    m = 2 if kernel in ("stokeslet", "stresslet") else 1
    err = 0.0
    for j in range(D, 3):
        Lj = geom.Lext[j]
        err = max(err, free_error_estimate(m, alpha, Lj, math.pi / Lj))
    return err <= tol
