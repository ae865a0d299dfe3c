"""The library's host-side plan tables (C++, dmk_plan_info / dmk_plan_table) against the oracle.

Both sides are FP64 and written independently from the paper (C++ std:: Bessel functions and
Sturm-bisection PSWF vs scipy and a dense eigensolver), so agreement is at roundoff.
No device is used.
"""
import numpy as np
import pytest

from oracle.dmk import root_parts
from oracle.kernels import Kernel
from oracle.params import Geometry, c_and_p, n_f, root_modes, TOL_ROWS
from oracle.pswf import PSWFWindow
from paper_2606_27134_b300 import dmk

GEOMS = [(3, [1, 1, 1]), (3, [1, 1, 16]), (2, [1, 1, 0.25]), (2, [1, 2, 1]), (1, [8, 1, 1]), (1, [1, 1, 1]),
         (0, [1, 1, 1]), (0, [0.5, 2, 1]),
         # free extents a few periods long: the original symbol for alpha != 0 (App. E switch)
         (2, [1, 1, 4]), (1, [1, 4, 3]), (2, [1.5, 1, 5])]


@pytest.mark.parametrize("kernel", ["laplace", "stokeslet", "stresslet", "rotlet"])
@pytest.mark.parametrize("tol", TOL_ROWS)
def test_parameters(kernel, tol):
    for D, L in GEOMS:
        info = dmk.plan_info(kernel, D, L, tol)
        c, p = c_and_p(kernel, tol)
        g = Geometry(D, L)
        assert info["c"] == pytest.approx(c, rel=1e-15) and info["p"] == p and info["n_f"] == n_f(c)
        assert info["M"] == list(g.M) and info["s"] == g.s
        parts = root_parts(Kernel(kernel), g, c, PSWFWindow(c), tol)
        assert info["n_root_modes"] == sum(int(pt[1].sum()) for pt in parts)
        kk, C, R, dk = root_modes(kernel, g, c)
        if D < 3:
            assert info["R"] == pytest.approx(R, rel=1e-15)


@pytest.mark.parametrize("kernel", ["laplace", "stokeslet", "stresslet", "rotlet"])
@pytest.mark.parametrize("D,L", GEOMS, ids=[f"{d}P-{l}" for d, l in GEOMS])
def test_root_weights(kernel, D, L):
    tol = 1e-6
    c, p = c_and_p(kernel, tol)
    g = Geometry(D, L)
    K = Kernel(kernel)
    parts = root_parts(K, g, c, PSWFWindow(c), tol)
    assert len(dmk.plan_table(kernel, D, L, tol, 5)) == (0 if len(parts) == 1 else sum(len(a) for a in parts[1][0]))
    for ip, (axes, keep, W, R) in enumerate(parts):
        ax = dmk.plan_table(kernel, D, L, tol, 5 * ip)
        n = [len(a) for a in axes]
        assert len(ax) == sum(n)
        assert np.allclose(ax, np.concatenate(axes), rtol=1e-15, atol=1e-15)
        w = dmk.plan_table(kernel, D, L, tol, 1 + 5 * ip)
        w = (w[0::2] + 1j * w[1::2]).reshape(n[0], n[1], n[2], K.d_u, K.d_rho)
        scale = np.max(np.abs(W))
        assert np.max(np.abs(w - W)) <= 1e-12 * scale


@pytest.mark.parametrize("kernel", ["laplace", "stokeslet", "stresslet", "rotlet"])
def test_difference_kernel_table(kernel):
    """Level-0 plane-wave symbol w_0 D_0-hat(h_0 m) (Eq. Dl_int_discr) on the half grid."""
    tol = 1e-6
    c, p = c_and_p(kernel, tol)
    nf = n_f(c)
    NF = 2 * nf + 1
    s = 1.0
    K = Kernel(kernel)
    win = PSWFWindow(c)
    h = 2 * np.pi / (3 * s)
    m = np.arange(-nf, nf + 1)
    mm = np.stack(np.meshgrid(m, m, np.arange(0, nf + 1), indexing="ij"), -1).reshape(-1, 3).astype(float)
    full = (h ** 3 / (2 * np.pi) ** 3) * K.diff_symbol(h * mm, s / 2, s, win)      # (n, du, drho)
    g = dmk.plan_table(kernel, 3, [1, 1, 1], tol, 2)
    assert len(g) == NF * NF * (nf + 1)
    lib = g[:, None, None] * K.op_symbol(mm)          # the library applies op(m) on integer m
    scale = np.max(np.abs(full))
    assert np.max(np.abs(lib - full)) <= 1e-12 * scale


@pytest.mark.parametrize("c_kernel", ["laplace", "stokeslet", "stresslet", "rotlet"])
@pytest.mark.parametrize("tol", TOL_ROWS)
def test_window_values(c_kernel, tol):
    c, p = c_and_p(c_kernel, tol)
    w = PSWFWindow(c)
    v = dmk.plan_table(c_kernel, 3, [1, 1, 1], tol, 3)
    d2phi = np.polynomial.legendre.legval(0.0, np.polynomial.legendre.legder(w.phi_coef, 2))
    assert v[0] == pytest.approx(w.phi0(), rel=1e-13)
    assert v[1] == pytest.approx(d2phi, rel=1e-11)
    assert v[2] == pytest.approx(w.d2phihat0(), rel=1e-11)
    assert np.allclose(v[3:], w.phihat(0.099 * c * np.arange(11)), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("kernel,tol", [("laplace", 1e-3), ("laplace", 1e-6), ("stokeslet", 1e-6),
                                        ("stresslet", 1e-6), ("rotlet", 1e-3), ("laplace", 1e-9)])
def test_residual_cubic_tables(kernel, tol):
    """FP32-path piecewise cubic tables of the residual series (App. B polynomial approximations)
    against the oracle's window: q = int_0^r phi / r, f = phi(r), g = phi'(r)/r in s = r^2, and
    their s-derivatives from the identities dq/ds = (f - q)/(2s), df/ds = g/2,
    dg/ds = (phi''(r) - g)/(2s).  The FP64 coefficients interpolate to 2e-8 of each series'
    scale (well below FP32 rounding); rounded to FP32 and evaluated in FP32 they stay within 4e-7."""
    from numpy.polynomial import legendre as npleg
    info = dmk.plan_info(kernel, 3, [1, 1, 1], tol)
    W = PSWFWindow(info["c"])
    NT = 256
    tab = dmk.plan_table(kernel, 3, [1, 1, 1], tol, 4).reshape(6, NT, 4)
    rng = np.random.default_rng(11)
    s = np.concatenate([rng.uniform(0.02, 1.0, 4000), [0.02, 0.5, 1.0 - 1e-12]])
    r = np.sqrt(s)
    I = 0.5 * (1.0 - W.Phi(r))                              # int_0^r phi
    q = I / r
    f = W.phi(r)
    g = W.dphi(r) / r
    d2 = npleg.legval(r, npleg.legder(W.phi_coef, 2))
    ref = [q, f, g, (f - q) / (2 * s), g / 2, (d2 - g) / (2 * s)]
    x = s * NT
    i = np.minimum(x.astype(int), NT - 1)
    u = x - i
    for k in range(6):
        c = tab[k, i]
        val = c[:, 0] + u * (c[:, 1] + u * (c[:, 2] + u * c[:, 3]))
        scale = np.max(np.abs(ref[k]))
        assert np.max(np.abs(val - ref[k])) <= 2e-8 * scale, k
        c32 = c.astype(np.float32)
        u32 = u.astype(np.float32)
        v32 = c32[:, 0] + u32 * (c32[:, 1] + u32 * (c32[:, 2] + u32 * c32[:, 3]))
        assert np.max(np.abs(v32.astype(np.float64) - ref[k])) <= 4e-7 * scale, k


# (D, L, the first root part's cube-index DFT lengths Q_a worked out by hand): a periodic axis of
# M_a cubes gives M_a (Sec. 3.4); a free axis of step pi/R gives 2 R / s when that is an integer
# (Sec. 5.4, Eq. kappaqdef): D = 2, L3 = 2 -> R = 3 s, Q3 = 6; L3 = 8 -> R = 9 s, Q3 = 18;
# D = 1, (L2, L3) = (2, 3) -> R = |(3, 4)| s = 5 s, Q = 10 on both free axes; |(2, 4)| s is not a
# rational multiple of s, a non-exact tiling and a single cube keep the direct sums (zeros)
DFT_GEOMS = [(3, [1, 1, 16], [1, 1, 16]), (3, [1, 3, 4], [1, 3, 4]), (3, [2, 3, 1], [2, 3, 1]),
             (2, [1, 3, 2], [1, 3, 6]), (2, [3, 1, 2], [3, 1, 6]), (2, [1, 1, 8], [1, 1, 18]),
             (1, [1, 2, 3], [1, 10, 10]), (1, [1, 1, 3], [0, 0, 0]), (3, [1, 1.3, 1.7], [0, 0, 0]),
             (2, [1, 1, 0.25], [0, 0, 0]), (0, [1, 2, 1], [0, 0, 0])]


@pytest.mark.parametrize("kernel", ["laplace", "stokeslet", "stresslet", "rotlet"])
@pytest.mark.parametrize("tol", [1e-3, 1e-6])
def test_cube_index_dft_lengths(kernel, tol):
    """Where the sums over the cubes become DFTs over the cube index, every wavenumber of every
    root part of the oracle is k = 2 pi n / (Q_a s) with consecutive integers n along each axis
    and Q_a >= M_a: the identity exp(-i k_a s m_a) = exp(-2 pi i (n mod Q_a) m_a / Q_a) behind
    Eqs. 1d-DFT-beta and beta_hat_oversampled then holds on the oracle's own grids."""
    for D, L, want in DFT_GEOMS:
        info = dmk.plan_info(kernel, D, L, tol)
        Q = info["root_dft_len"]
        assert Q[0] == want, (D, L, Q)
        c, _ = c_and_p(kernel, tol)
        g = Geometry(D, L)
        parts = root_parts(Kernel(kernel), g, c, PSWFWindow(c), tol)
        if want == [0, 0, 0]:
            assert Q[1] == [0, 0, 0]
            continue
        assert Q[1] == ([0, 0, 0] if len(parts) == 1 else Q[1]) and (len(parts) == 1 or min(Q[1]) >= 1)
        for ip, (axes, *_rest) in enumerate(parts):
            for a in range(3):
                if g.M[a] == 1 or (len(axes[a]) == 1 and axes[a][0] == 0.0):
                    assert Q[ip][a] == 1        # one cube, or only k = 0: every phase is 1
                    continue
                assert Q[ip][a] >= g.M[a]
                n = np.asarray(axes[a]) * Q[ip][a] * g.s / (2 * np.pi)
                assert np.max(np.abs(n - np.rint(n))) < 1e-9, (D, L, ip, a)
                if len(n) > 1:
                    assert np.all(np.diff(np.rint(n)) == 1)


@pytest.mark.parametrize("kernel,D,L", [("laplace", 3, [1, 3, 4]), ("rotlet", 3, [2, 3, 1]), ("laplace", 2, [1, 3, 2]),
                                        ("laplace", 2, [1, 1, 8]), ("stokeslet", 1, [1, 2, 3]),
                                        ("rotlet", 2, [1, 1, 3])],
                         ids=["3P-1x3x4", "3P-2x3x1", "2P-1x3x2", "2P-1x1x8", "1P-1x2x3", "2P-1x1x3"])
def test_cube_index_dft_reproduces_direct_sums(kernel, D, L):
    """The sums over the cubes of Eqs. structurefac and eval_tensor, written as a zero-padded FFT
    over the cube index at the plan's lengths Q_a (Eqs. 1d-DFT-beta and beta_hat_oversampled:
    beta-hat_s = sum_m exp(-2 pi i s . m / Q) rho~^m, chi(k) = exp(-i k . c_0) sum_j S(j, k)
    beta-hat_{n(k) mod Q}(j); the evaluation by the inverse FFT of the sums grouped by n mod Q),
    equal the direct sums over the cubes with the oracle's own root parts and nodes, for random
    root proxies: the lengths of the library's plan and the reading of Sec. 3.4 and 5.4 together
    reproduce the definition.  numpy's FFT, no device."""
    from oracle.dmk import cheb_nodes
    tol = 1e-3
    K = Kernel(kernel)
    c, p = c_and_p(kernel, tol)
    g = Geometry(D, L)
    Q = dmk.plan_info(kernel, D, L, tol)["root_dft_len"]
    parts = root_parts(K, g, c, PSWFWindow(c), tol)
    assert min(Q[0]) >= 1 and (len(parts) == 1 or min(Q[1]) >= 1)
    M = list(g.M)
    y = (g.s / 2) * cheb_nodes(p)
    rng = np.random.default_rng(17)
    prox = rng.standard_normal((M[0], M[1], M[2], p, p, p, K.d_rho))        # [m1, m2, m3, j1, j2, j3, a]
    cen = [(np.arange(M[a]) + 0.5) * g.s for a in range(3)]
    c0 = 0.5 * g.s
    for ip, (axes, keep, Wk, _) in enumerate(parts):
        S = [np.exp(-1j * np.outer(ax, y)) for ax in axes]                  # S[a][i, j] = exp(-i k y_j)
        E = [np.exp(-1j * np.outer(cen[a], axes[a])) for a in range(3)]     # E[a][m, i] = exp(-i k c_m)
        chi_dir = np.einsum("xa,yb,zc,ai,bj,ck,xyzijkd->abcd", E[0], E[1], E[2], S[0], S[1], S[2], prox,
                            optimize=True)
        u_hat = np.einsum("abcud,abcd->abcu", Wk, chi_dir)
        u_dir = np.einsum("xa,yb,zc,ai,bj,ck,abcu->xyzijku", E[0].conj(), E[1].conj(), E[2].conj(), S[0].conj(),
                          S[1].conj(), S[2].conj(), u_hat, optimize=True).real
        q = Q[ip]
        # the group of every wavenumber: n mod Q_a with k = 2 pi n / (Q_a s)
        P = []
        for a in range(3):
            n = np.rint(np.asarray(axes[a]) * q[a] * g.s / (2 * np.pi)).astype(np.int64)
            P.append((np.mod(n, q[a])[None, :] == np.arange(q[a])[:, None]).astype(float))   # [s, i]
        bhat = np.fft.fftn(prox, s=q, axes=(0, 1, 2))                       # zero padded from M to Q
        ph0 = np.exp(-1j * c0 * (axes[0][:, None, None] + axes[1][None, :, None] + axes[2][None, None, :]))
        chi_dft = ph0[..., None] * np.einsum("xa,yb,zc,ai,bj,ck,xyzijkd->abcd", P[0], P[1], P[2], S[0], S[1], S[2],
                                             bhat, optimize=True)
        scale = np.max(np.abs(chi_dir))
        assert np.max(np.abs(chi_dft - chi_dir)) <= 1e-12 * scale, (ip, q)
        G = np.einsum("xa,yb,zc,ai,bj,ck,abcu->xyzijku", P[0], P[1], P[2], S[0].conj(), S[1].conj(), S[2].conj(),
                      ph0.conj()[..., None] * u_hat, optimize=True)
        u_dft = (np.prod(q) * np.fft.ifftn(G, axes=(0, 1, 2)))[:M[0], :M[1], :M[2]].real
        assert np.max(np.abs(u_dft - u_dir)) <= 1e-12 * np.max(np.abs(u_dir)), (ip, q)
