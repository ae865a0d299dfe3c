"""The periodized DMK evaluation, step by step (oracle; test infrastructure only).

Sec. 3.1 gives the five steps (octree, upward pass, top level, downward pass, leaf);
Sec. 4.2 runs them on the forest of cubes; Sec. 4.3 (Eqs. structurefacgen,
ufar_chebgrid, eval_tensor, structurefac) and Sec. 5.3 (Eq. ewald_far_allP_discr with
the truncated symbols of Sec. 5.2 and App. C-D) give the root far field; Sec. 2.3
(Eqs. u_diff_l, Dl_int_discr) the plane-wave difference-kernel sums; Sec. 2.4 the self
correction.  Readings where the paper is silent are stated next to the code.

Gradients with respect to the target position are taken by complex-step
differentiation of the same expressions (Im f(x + i h e_i)/h), so they are exact
derivatives of the computed approximation u(x_t).
"""
import math
import numpy as np

from .params import c_and_p, n_f, Geometry, root_modes, original_symbol_ok, free_count
from .pswf import PSWFWindow
from .kernels import Kernel
from .tree import BITS, Forest, wrap, replicate, quantize
from . import symbols as sym

_CSTEP = 1e-30


def cheb_nodes(p):
    """First-kind Chebyshev points eta_j = cos((2j-1) pi/(2p)), j=1..p (Sec. 3.1.2)."""
    j = np.arange(1, p + 1)
    return np.cos((2 * j - 1) * np.pi / (2 * p))


def lagrange(x, nodes):
    """Lagrange basis l_j(x) = prod_{k != j} (x - eta_k)/(eta_j - eta_k); shape (len(x), p).

    Product form, valid for complex x (used for complex-step gradients).
    """
    x = np.asarray(x)
    p = len(nodes)
    out = np.ones((x.shape[0], p), dtype=np.result_type(x, np.float64))
    for j in range(p):
        for k in range(p):
            if k != j:
                out[:, j] = out[:, j] * (x - nodes[k]) / (nodes[j] - nodes[k])
    return out


def root_symbol(kern, geom, c, win):
    """Root far-field weights C^{DP} G-hat(k) gamma-hat(|k| nu_0) for every retained mode.

    D=3: G-hat = D-hat(k)/|k|^{2,4} (Eq. ewald_far_3P; App. B).
    D=2: for (k1,k2) != 0, D-hat(k) A-hat_1^{alpha,R}(|k3|) with alpha = |(k1,k2)|; for
         (k1,k2) = 0 the zero-mode forms of App. D (Laplace H-hat_1^{0,R}; Stokeslet
         C^E H-hat_1^{0,R}; stresslet and rotlet C^E Z-hat_1^{0,R}) -- Eq. ewald_far_es_2P_discr_a.
    D=1: for k1 != 0, D-hat(k) A-hat_2^{|k1|,R}(kappa); for k1 = 0, C^H H-hat_2^{0,R} + C^B B-hat_2^{0,R}
         (App. D); truncated symbols for every k1 (Remark alpha_switch).
    D=0: D-hat(k) A-hat_3^R(|k|) with the truncated kernels of symbols.H3_trunc / B3_trunc.
    Returns (axes, keep, W, R): W on the wavenumber rectangle, shape (n1, n2, n3, d_u, d_rho),
    zero outside the retained set.
    """
    axes, keep, C, R, dk = root_modes(kern.name, geom, c, return_axes=True)
    shp = keep.shape
    kk = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    kk[~keep.ravel()] = 0.0       # dropped modes: evaluated at k = 0 below, then zeroed
    kn = np.sqrt(np.sum(kk * kk, axis=1))
    gam = kern.screening(kn * geom.nu0, win)
    D = geom.D
    n = kk.shape[0]
    W = np.zeros((n, kern.d_u, kern.d_rho), dtype=complex)
    bih = kern.biharmonic
    if D == 3:
        with np.errstate(divide="ignore", invalid="ignore"):
            W = kern.op_symbol(kk) / (kn ** (4 if bih else 2))[:, None, None]
    elif D == 0:
        A = sym.B3_trunc(kn, R) if bih else sym.H3_trunc(kn, R)
        W = kern.op_symbol(kk) * A[:, None, None]
    elif D == 2:
        alpha = np.sqrt(kk[:, 0] ** 2 + kk[:, 1] ** 2)
        k3 = kk[:, 2]
        nz = alpha > 0
        A = sym.B1_trunc(alpha[nz], k3[nz], R) if bih else sym.H1_trunc(alpha[nz], k3[nz], R)
        W[nz] = kern.op_symbol(kk[nz]) * A[:, None, None]
        z = ~nz
        if np.any(z):
            W[z] = _zero_mode_2p(kern, k3[z], R)
    elif D == 1:
        alpha = np.abs(kk[:, 0])
        kap = np.sqrt(kk[:, 1] ** 2 + kk[:, 2] ** 2)
        nz = alpha > 0
        A = sym.B2_trunc(alpha[nz], kap[nz], R) if bih else sym.H2_trunc(alpha[nz], kap[nz], R)
        W[nz] = kern.op_symbol(kk[nz]) * A[:, None, None]
        z = ~nz
        if np.any(z):
            W[z] = _zero_mode_1p(kern, kk[z, 1], kk[z, 2], R)
    W[~keep.ravel()] = 0.0
    W = C * W * gam[:, None, None]
    return axes, keep, W.reshape(shp + (kern.d_u, kern.d_rho)), R


def root_parts(kern, geom, c, win, tol):
    """The root far field as one or two wavenumber rectangles, each (axes, keep, W, R) as
    root_symbol returns them; their contributions add.

    Truncated symbol for every mode (Remark alpha_switch), unless the App. E switch
    (params.original_symbol_ok) allows the original one: then the alpha != 0 modes take the
    original mollified symbol D-hat(k) gamma-hat(|k| nu_0)/|k|^{2,4} on the free grid of step
    pi/L_j (the Nyquist step of the original kernel, Sec. 5.3) with the constant C^{DP} of that
    step, and the alpha = 0 modes keep the truncated zero-mode symbols on the step-pi/R grid
    (Eq. ewald_far_es_1P_discr_b, and its D = 2 analogue).
    """
    if not original_symbol_ok(kern.name, geom, tol):
        return [root_symbol(kern, geom, c, win)]
    D = geom.D
    axes_t, keep_t, W_t, R = root_symbol(kern, geom, c, win)
    # part 1: the alpha = 0 line of the truncated rectangle
    sl = tuple(slice(int(np.argmin(np.abs(axes_t[i]))), int(np.argmin(np.abs(axes_t[i]))) + 1) if i < D
               else slice(None) for i in range(3))
    axes_z = [axes_t[i][sl[i]] for i in range(3)]
    part_z = (axes_z, keep_t[sl], W_t[sl], R)
    # part 2: alpha != 0 with the original symbol
    K = c / geom.nu0
    axes_o = []
    steps = []
    for i in range(3):
        if i < D:
            axes_o.append(axes_t[i])
        else:
            h = math.pi / geom.Lext[i]
            n = free_count(K, h)
            axes_o.append(h * np.arange(-n, n + 1))
            steps.append(h)
    kk = np.stack(np.meshgrid(*axes_o, indexing="ij"), axis=-1).reshape(-1, 3)
    kn = np.sqrt(np.sum(kk * kk, axis=1))
    alpha = np.sqrt(np.sum(kk[:, :D] ** 2, axis=1))
    keep = (kn * geom.nu0 <= c * (1 + 1e-12)) & (alpha > 0)
    kk[~keep] = 1.0              # dropped modes: a harmless point, zeroed below
    kn = np.sqrt(np.sum(kk * kk, axis=1))
    W = kern.op_symbol(kk) * (kern.screening(kn * geom.nu0, win) / kn ** (4 if kern.biharmonic else 2))[:, None, None]
    W[~keep] = 0.0
    if D == 2:
        C = steps[0] / (geom.L[0] * geom.L[1] * 2 * math.pi)
    else:
        C = steps[0] * steps[1] / (geom.L[0] * (2 * math.pi) ** 2)
    shp = tuple(len(a) for a in axes_o)
    part_o = (axes_o, keep.reshape(shp), (C * W).reshape(shp + (kern.d_u, kern.d_rho)), R)
    return [part_z, part_o]


def _zero_mode_2p(kern, k3, R):
    """(k1,k2) = (0,0) symbols of App. D (Eqs. C_stokeslet_rotlet_E_2p, C_stresslet_E_2p)."""
    n = k3.shape[0]
    kap = np.abs(k3)
    if kern.name == "laplace":
        return sym.H1_trunc(0.0, kap, R).reshape(n, 1, 1).astype(complex)
    if kern.name == "stokeslet":
        CE = np.diag([1.0, 1.0, 0.0])
        return CE[None] * sym.H1_trunc(0.0, kap, R)[:, None, None]
    Z = sym.Z1_trunc(k3, R)
    if kern.name == "rotlet":
        CE = np.array([[0.0, 1.0, 0.0], [-1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
        return CE[None] * Z[:, None, None]
    # stresslet: C_j^E as matrices in (l, m)
    CE = np.zeros((3, 3, 3))
    CE[0] = [[0, 0, -2], [0, 0, 0], [-2, 0, 0]]
    CE[1] = [[0, 0, 0], [0, 0, -2], [0, -2, 0]]
    CE[2] = [[-2, 0, 0], [0, -2, 0], [0, 0, -2]]
    return CE.reshape(1, 3, 9) * Z[:, None, None]


def _zero_mode_1p(kern, k2, k3, R):
    """k1 = 0 symbols of App. D: C^H H-hat_2^{0,R}(kappa) + C^B B-hat_2^{0,R}(kappa)."""
    n = k2.shape[0]
    kap = np.sqrt(k2 ** 2 + k3 ** 2)
    H = sym.H2_trunc(0.0, kap, R)
    if kern.name == "laplace":
        return H.reshape(n, 1, 1).astype(complex)
    B = sym.B2_trunc(0.0, kap, R)
    out = np.zeros((n, 3, kern.d_rho), dtype=complex)
    if kern.name == "stokeslet":
        out[:, 0, 0] = H
        out[:, 1, 1] = k3 ** 2 * B
        out[:, 1, 2] = -k2 * k3 * B
        out[:, 2, 1] = -k2 * k3 * B
        out[:, 2, 2] = k2 ** 2 * B
        return out
    if kern.name == "rotlet":
        CH = np.zeros((n, 3, 3))
        CH[:, 0, 1] = k3
        CH[:, 0, 2] = -k2
        CH[:, 1, 0] = -k3
        CH[:, 2, 0] = k2
        return -0.5j * CH * H[:, None, None]
    # stresslet: C_j^H = i Ct_j^H, C_j^B = i Ct_j^B, matrices in (l, m)
    kq = kap ** 2
    CtH = np.zeros((n, 3, 3, 3))
    CtH[:, 0, 0, 1] = k2
    CtH[:, 0, 0, 2] = k3
    CtH[:, 0, 1, 0] = k2
    CtH[:, 0, 2, 0] = k3
    CtH[:, 1, 0, 0] = k2
    CtH[:, 2, 0, 0] = k3
    CtB = np.zeros((n, 3, 3, 3))
    CtB[:, 1, 1, 1] = k2 * (3 * kq - 2 * k2 ** 2)
    CtB[:, 1, 1, 2] = k3 * (kq - 2 * k2 ** 2)
    CtB[:, 1, 2, 1] = k3 * (kq - 2 * k2 ** 2)
    CtB[:, 1, 2, 2] = k2 * (kq - 2 * k3 ** 2)
    CtB[:, 2, 1, 1] = k3 * (kq - 2 * k2 ** 2)
    CtB[:, 2, 1, 2] = k2 * (kq - 2 * k3 ** 2)
    CtB[:, 2, 2, 1] = k2 * (kq - 2 * k3 ** 2)
    CtB[:, 2, 2, 2] = k3 * (3 * kq - 2 * k3 ** 2)
    T = 1j * (CtH * H[:, None, None, None] + CtB * B[:, None, None, None])
    return T.reshape(n, 3, 9)


class Result:
    pass


def evaluate(kernel, D, L, tol, points, strengths, n_s=250, grad=False, return_parts=False, targets=None,
             owned_cubes=None, chi_reduce=None):
    """Evaluate u(x_t) = sum_s sum*_p K(x_t - x_s + p) rho_s (Eq. periodic_sum) by periodized DMK.

    points (N,3), strengths (N, d_rho); returns potentials (N, d_u) in input order and, if
    grad, the target gradients g[t, i, j] = d u_j / d x_i (N, 3, d_u).

    targets: None (every point is a target) or an array of point indices.  The method is the
    same -- every point is a source, the forest, upward pass, root far field and downward pass
    are those of the whole problem -- but the leaf step (Sec. 3.1.5) runs only for the listed
    targets, so each of their values is the one the full evaluation gives; the other rows of
    the outputs are NaN.

    owned_cubes, chi_reduce: the spatial split of the evaluation over several evaluators.  The
    structure factor of Eq. structurefac is a sum over the cubes; with owned_cubes (cube indices
    m1 + M1 (m2 + M2 m3)) only those cubes enter this evaluator's partial sum, and
    chi_reduce(partial) -> total combines the partial sums of all evaluators (e.g. an
    all-reduce): it receives one flat complex vector, the structure factor (of each root part
    in turn, see root_parts) followed by the d_rho strength sums over the own cubes (the total strength enters the Stokeslet constants).  The points given are then this evaluator's own points plus those of the
    cubes adjacent to its own cubes (the near field of Sec. 3.1.4-3.1.5 reaches no further),
    and targets should be its own points.
    """
    kern = Kernel(kernel)
    c, p = c_and_p(kernel, tol)
    geom = Geometry(D, L)
    win = PSWFWindow(c)
    nf = n_f(c)
    x = np.asarray(points, dtype=np.float64)
    N = x.shape[0]
    rho = np.asarray(strengths, dtype=np.float64).reshape(N, kern.d_rho)
    if kernel == "laplace" and D in (1, 2) and abs(rho.sum()) > 1e-12 * max(np.abs(rho).sum(), 1e-300):
        raise ValueError("Laplace with D=1,2 requires zero net charge (Sec. 5.2)")
    # wrapped points, then (non-exact tilings, Sec. 4.1.2) the periodic images that fall in
    # Omega_ext as extra sources: points N.. of w, with src mapping every point to its original
    w, src = replicate(wrap(x, geom), geom)
    rho_t = rho                      # the targets' strengths
    rho = rho[src]                   # every source's strength, images included
    G = quantize(w, geom)
    forest = Forest(geom, G, n_s)
    boxes = forest.by_id
    nb = len(boxes)
    nodes = cheb_nodes(p)
    s = geom.s

    def center(b):
        r = s / 2 ** b.level
        return np.array([geom.origin[i] + (b.ix[i] + 0.5) * r for i in range(3)])

    # ---- step 2: upward pass (Sec. 3.1.2, 4.2) -----------------------------------
    proxy = [None] * nb
    # child-in-parent interpolation: child node eta_j sits at (2o-1)/2 + eta_j/2 in parent units
    Ioct = [lagrange((2 * o - 1) / 2 + nodes / 2, nodes) for o in (0, 1)]   # [j_child, j_parent]
    for b in sorted(boxes, key=lambda b: -b.level):
        if b.is_leaf:
            pr = np.zeros((p, p, p, kern.d_rho))
            if len(b.pts):
                xi = (w[b.pts] - center(b)) / (s / 2 ** b.level / 2)
                Lx, Ly, Lz = (lagrange(xi[:, i], nodes) for i in range(3))
                pr = np.einsum("sa,sb,sc,sd->abcd", Lx, Ly, Lz, rho[b.pts], optimize=True)
            proxy[b.id] = pr
        else:
            pr = np.zeros((p, p, p, kern.d_rho))
            for ch in b.children:
                o = [ch.ix[i] - 2 * b.ix[i] for i in range(3)]
                pr += np.einsum("abcd,aA,bB,cC->ABCd", proxy[ch.id], Ioct[o[0]], Ioct[o[1]], Ioct[o[2]],
                                optimize=True)
            proxy[b.id] = pr

    # ---- step 3: root far field (Sec. 3.1.3, 4.3, 5.3) ---------------------------
    # Tensor-product form of Eqs. structurefac and eval_tensor on the rectangle of
    # wavenumbers enclosing the retained set; dropped modes carry weight zero.
    local = [None] * nb
    parts = root_parts(kern, geom, c, win, tol)
    R = parts[0][3]
    roots = forest.roots
    y = (s / 2) * nodes

    def chi_proxy(b):
        """The root proxy charges entering the structure factor: only sources inside Omega count
        (Sec. 4.3, non-exact tilings).  A cube inside Omega gives its proxy; a padding cube
        outside Omega gives nothing; a cut cube gives its original sources (not their images),
        anterpolated directly onto its root grid (the paper sums the proxies of its uncut
        descendants plus the sources of its cut leaves; the grid of the cube itself represents
        the same band-limited modes)."""
        inside, outside = True, False
        for i in range(3):
            if geom.padded[i]:
                lo = geom.origin[i] + b.ix[i] * s
                if lo >= geom.L[i] or lo + s <= 0.0:
                    outside = True
                if lo < 0.0 or lo + s > geom.L[i]:
                    inside = False
        if outside:
            return None
        if inside:
            return proxy[b.id]
        orig = b.pts[b.pts < N]
        if not len(orig):
            return None
        xi = (w[orig] - center(b)) / (s / 2)
        Lx, Ly, Lz = (lagrange(xi[:, i], nodes) for i in range(3))
        return np.einsum("sa,sb,sc,sd->abcd", Lx, Ly, Lz, rho[orig], optimize=True)

    Mc = geom.M

    def cube_index(b):
        return b.ix[0] + Mc[0] * (b.ix[1] + Mc[1] * b.ix[2])

    owned = None if owned_cubes is None else set(int(m) for m in owned_cubes)
    # total strength, for the constants of Sec. 5 that multiply it (the truncated Stokeslet,
    # Remark stokeslet_const_corr): over this evaluator's own cubes when split, then reduced
    # with the structure factor
    rho_sum = rho_t.sum(axis=0)
    if owned is not None:
        Go = G[:N] >> BITS
        mine = np.isin(Go[:, 0] + Mc[0] * (Go[:, 1] + Mc[1] * Go[:, 2]), sorted(owned))
        rho_sum = rho_t[mine].sum(axis=0)
    proxies = {}
    for b in roots:
        if owned is not None and cube_index(b) not in owned:
            continue
        pr = chi_proxy(b)
        if pr is not None:
            proxies[b.id] = pr
    chis, Scs = [], []
    for axes, keep, Wk, _ in parts:
        Sc = [np.exp(-1j * np.outer(ax, y)) for ax in axes]            # conj(S(j, k)) [k, j]
        chi = np.zeros(keep.shape + (kern.d_rho,), dtype=complex)
        for b in roots:
            if b.id not in proxies:
                continue
            cb = center(b)
            ph = np.exp(-1j * (axes[0][:, None, None] * cb[0] + axes[1][None, :, None] * cb[1]
                               + axes[2][None, None, :] * cb[2]))
            chi += ph[..., None] * np.einsum("ai,bj,ck,ijkd->abcd", Sc[0], Sc[1], Sc[2], proxies[b.id],
                                             optimize=True)
        chis.append(chi)
        Scs.append(Sc)
    if chi_reduce is not None:
        flat = chi_reduce(np.concatenate([ch.ravel() for ch in chis] + [rho_sum.astype(complex)]))
        o = 0
        for i, ch in enumerate(chis):
            chis[i] = flat[o:o + ch.size].reshape(ch.shape)
            o += ch.size
        rho_sum = flat[o:].real
    for b in roots:
        local[b.id] = 0.0
    for (axes, keep, Wk, _), chi, Sc in zip(parts, chis, Scs):
        uhat = np.einsum("abcud,abcd->abcu", Wk, chi)
        for b in roots:
            cb = center(b)
            ph = np.exp(1j * (axes[0][:, None, None] * cb[0] + axes[1][None, :, None] * cb[1]
                              + axes[2][None, None, :] * cb[2]))
            local[b.id] = local[b.id] + np.einsum("ai,bj,ck,abcu->ijku", Sc[0].conj(), Sc[1].conj(), Sc[2].conj(),
                                                  ph[..., None] * uhat, optimize=True).real
    if kernel == "stokeslet" and D == 0:
        # constant removed by the C^1 gauge of the truncated biharmonic kernel (symbols.B3_trunc)
        cst = sym.stokeslet_free_space_constant(R) * rho_sum
        for b in roots:
            local[b.id] = local[b.id] + cst

    # ---- step 4: downward pass (Sec. 3.1.4, Eq. Dl_int_discr) --------------------
    pw, direct = forest.interactions()
    mvec = np.arange(-nf, nf + 1)
    for l in range(forest.nlevels):
        nul = s / 2 ** l
        h = 2 * np.pi / (3 * nul)                 # h_l = 2 pi/(3 nu_l) (Sec. 2.3)
        if pw[l]:
            mm = np.stack(np.meshgrid(mvec, mvec, mvec, indexing="ij"), axis=-1).reshape(-1, 3)
            sym_l = (h ** 3 / (2 * np.pi) ** 3) * kern.diff_symbol(h * mm, nul / 2, nul, win)
            NF = len(mvec)
            yrel = (nul / 2) * nodes
            Eout = np.exp(-1j * h * np.outer(mvec, yrel))    # [m, j]
            Ein = np.exp(1j * h * np.outer(mvec, yrel))
            Wout = {}
            V = {}
            for (A, S, sh) in pw[l]:
                if S.id not in Wout:
                    Wout[S.id] = np.einsum("ai,bj,ck,ijkd->abcd", Eout, Eout, Eout, proxy[S.id], optimize=True)
                img = center(S) + np.array(sh) * np.array(geom.L)
                ph = np.exp(1j * h * (mm @ (center(A) - img))).reshape(NF, NF, NF, 1)
                V[A.id] = V.get(A.id, 0) + ph * Wout[S.id]
            for aid, v in V.items():
                vu = np.einsum("mab,mb->ma", sym_l, v.reshape(-1, kern.d_rho)).reshape(NF, NF, NF, kern.d_u)
                local[aid] = local[aid] + np.einsum("ai,bj,ck,abcd->ijkd", Ein, Ein, Ein, vu,
                                                    optimize=True).real
        # shift (interpolate) every non-leaf grid at level l to its children
        for b in boxes:
            if b.level == l and not b.is_leaf:
                for ch in b.children:
                    o = [ch.ix[i] - 2 * b.ix[i] for i in range(3)]
                    local[ch.id] = np.einsum("abcd,Aa,Bb,Cc->ABCd", local[b.id], Ioct[o[0]], Ioct[o[1]],
                                             Ioct[o[2]], optimize=True)

    # ---- step 5: leaf evaluation, residual sums, self correction (Sec. 3.1.5, 2.4) --
    u = np.zeros((N, kern.d_u))
    gu = np.zeros((N, 3, kern.d_u)) if grad else None
    want = None
    if targets is not None:
        want = np.zeros(N, dtype=bool)
        want[np.asarray(targets, dtype=np.int64)] = True
        u[:] = np.nan
        if grad:
            gu[:] = np.nan
    per_leaf = {}
    for (A, S, sh, l) in direct:
        for T in forest.leaves_below(A):
            if len(T.pts):
                per_leaf.setdefault(T.id, []).append((S, sh, l))
    Lvec = np.array(geom.L)
    for T in forest.leaves():
        t = T.pts[T.pts < N]                       # original points only are targets
        if want is not None:
            t = t[want[t]]
        if not len(t):
            continue
        cT = center(T)
        half = s / 2 ** T.level / 2

        def cheb_val(xt):
            xi = (xt - cT) / half
            Lx, Ly, Lz = (lagrange(xi[:, i], nodes) for i in range(3))
            return np.einsum("ta,tb,tc,abcd->td", Lx, Ly, Lz, local[T.id], optimize=True)

        def resid(xt):
            acc = np.zeros((len(t), kern.d_u), dtype=xt.dtype)
            for (S, sh, l) in per_leaf.get(T.id, []):
                srcs = forest_points_below(S)
                if not len(srcs):
                    continue
                nul = s / 2 ** l
                img = w[srcs] + np.array(sh) * Lvec
                dx = xt[:, None, :] - img[None, :, :]              # (nt, ns, 3)
                r2 = np.sum(dx.real ** 2, axis=2)
                # excluded: r = 0 (p = 0 with x_t = x_s, Eq. periodic_sum) and the target's own
                # periodic images, which lie at |p| >= min periodic L_i = nu_0 >= nu, outside the
                # support of K_R whatever the rounding of r^2 (Remark comp_supp)
                ok = (r2 < nul * nul) & (r2 > 0) & (src[srcs][None, :] != t[:, None])
                ti, si = np.nonzero(ok)
                if len(ti) == 0:
                    continue
                K = kern.residual(dx[ti, si], nul, win)             # (npairs, d_u, d_rho)
                contrib = np.einsum("nab,nb->na", K, rho[srcs][si])
                np.add.at(acc, ti, contrib)
            return acc

        def total(xt):
            return cheb_val(xt) + resid(xt)

        ut = total(w[t]).real
        selfm = kern.self_matrix(s / 2 ** T.level, win)
        u[t] = ut - rho_t[t] @ selfm.T
        if grad:
            for i in range(3):
                xc = w[t].astype(complex)
                xc[:, i] += 1j * _CSTEP
                gu[t, i, :] = total(xc).imag / _CSTEP
            gu[t] -= np.einsum("ija,ta->tij", kern.self_grad(s / 2 ** T.level, win), rho_t[t])

    # 1P Stokeslet constant (Remark stokeslet_const_corr)
    if kernel == "stokeslet" and D == 1:
        Rr = R
        corr = -np.diag([(1 + math.log(Rr)) / (2 * np.pi), (math.log(Rr) + 0.5) / (4 * np.pi),
                         (math.log(Rr) + 0.5) / (4 * np.pi)]) / geom.L[0]
        u += (corr @ rho_sum)[None, :]    # NaN rows (targets not evaluated) stay NaN
    res = Result()
    res.u = u
    res.grad = gu
    res.forest = forest
    res.local = local
    res.proxy = proxy
    res.plan = dict(c=c, p=p, nf=nf, nmodes=sum(int(pt[1].sum()) for pt in parts), nparts=len(parts), R=R,
                    nlevels=forest.nlevels)
    return res


def forest_points_below(b):
    """Indices of all points in the subtree of box b (they are exactly b.pts)."""
    return b.pts


def evaluate_targets(kernel, D, L, tol, sources, strengths, targets, n_s=250, grad=False):
    """Eq. periodic_sum at a target set apart from the sources:
    u(y_t) = sum_s sum*_p K(y_t - x_s + p) rho_s, the terms with y_t - x_s + p = 0 skipped.

    The forest is built on sources and targets together, the targets entering as points of
    zero strength: they add nothing to any proxy, plane wave or residual sum, their self term
    (their own strength times K_M(0)) is zero, and the leaf step (Sec. 3.1.5) runs for them
    only.  Returns a Result with u (M, d_u) and, if grad, grad (M, 3, d_u).
    """
    kern = Kernel(kernel)
    y = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    x = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
    M = y.shape[0]
    rho = np.asarray(strengths, dtype=np.float64).reshape(x.shape[0], kern.d_rho)
    pts = np.vstack([y, x])
    q = np.vstack([np.zeros((M, kern.d_rho)), rho])
    r = evaluate(kernel, D, L, tol, pts, q, n_s=n_s, grad=grad, targets=np.arange(M))
    out = Result()
    out.u = r.u[:M]
    if grad:
        out.grad = r.grad[:M]
    return out
