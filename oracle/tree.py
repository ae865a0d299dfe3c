"""Forest of octrees and the DMK interaction structure (oracle; test infrastructure only).

Sec. 3.1.1: boxes split into 8 children while they hold more than n_s points; the
tree is then made level-restricted (2:1 balanced: leaves sharing a boundary point
differ by at most one level), with neighbour relations extended by periodic
wrapping.  Sec. 4.1.3: one octree per cube of the tiling, neighbour lists across
cubes, periodicity in the exactly tiled directions, balance over the whole forest; a direction
that is periodic but not exactly tiled is padded and non-periodic in the forest (Sec. 4.1.1,
4.1.2), its periodic images being extra sources (replicate()).

Membership is decided on integer coordinates: a point's global integer coordinate
on the finest grid (BITS levels below the cube) is G_i = floor((w_i / s) 2^BITS)
clamped to the tiled axis, where w is the (wrapped) coordinate and s the cube side.
A box at level l with integer index ix on axis i holds the points with
G_i >> (BITS - l) == ix.  Ties therefore go to the upper child.

The interaction structure follows the multilevel telescoping split (Eqs.
multilevel_ks, diffkernel, u_four_partsDP): for two colleague boxes (same level,
sharing a boundary point, including periodic images) K_R(nu_l) between their points
equals D_l + K_R(nu_{l+1}).  When both boxes have children, D_l is evaluated by plane
waves (Sec. 3.1.4) and the K_R(nu_{l+1}) remainder recurses into colleague child
pairs (non-colleague children are farther apart than nu_{l+1}, where K_R vanishes,
Remark comp_supp).  When either box is a leaf, K_R(nu_l) is summed directly between
the leaves below the target box and the points below the source box (Sec. 3.1.5).
"""
import itertools
import numpy as np

BITS = 18          # finest integer level below a cube; also the depth cap


def wrap(points, geom):
    """Wrap periodic coordinates into [0, L_i) (Eq. periodic-images).

    Periodic axis: w = x - L floor(x/L); w >= L -> w - L; w < 0 -> 0.
    Free axis: w = x, which must lie in [0, L_i) (else ValueError).
    """
    x = np.asarray(points, dtype=np.float64)
    w = np.empty_like(x)
    for i in range(3):
        Li = geom.L[i]
        if geom.periodic[i]:
            wi = x[:, i] - Li * np.floor(x[:, i] / Li)
            wi = np.where(wi >= Li, wi - Li, wi)
            wi = np.where(wi < 0, 0.0, wi)
        else:
            wi = x[:, i].copy()
            if np.any(~(wi >= 0)) or np.any(~(wi < Li)):
                raise ValueError("point outside the free extent [0, L_i)")
        w[:, i] = wi
    return w


def replicate(w, geom):
    """Periodic images of the sources in the padded (non-exactly tiled) directions (Sec. 4.1.2).

    Every image w + sum_i n_i L_i e_i (n_i integer, n = 0 excluded, i over the padded axes)
    that falls inside Omega_ext = [origin_i, origin_i + M_i s) is added.  Returns (w_ext, src):
    the original points first, then the images in order of (n, source); src[j] is the index of
    the original point behind point j.
    """
    N = w.shape[0]
    axes = [i for i in range(3) if geom.padded[i]]
    if not axes:
        return w, np.arange(N)
    pts, src = [w], [np.arange(N)]
    lo = np.array(geom.origin)
    hi = lo + np.array(geom.M) * geom.s
    rng = range(-3, 4)
    for ns in itertools.product(rng, repeat=len(axes)):
        if all(n == 0 for n in ns):
            continue
        img = w.copy()
        for i, n in zip(axes, ns):
            img[:, i] = w[:, i] + n * geom.L[i]
        inside = np.all((img >= lo) & (img < hi), axis=1)
        pts.append(img[inside])
        src.append(np.nonzero(inside)[0])
    return np.vstack(pts), np.concatenate(src)


def quantize(w, geom):
    """Global integer coordinates G = floor(((w - origin) / s) * 2^BITS), clamped to
    [0, M_i 2^BITS - 1]; the origin is the lower corner of Omega_ext (0 unless padded)."""
    G = np.empty(w.shape, dtype=np.int64)
    for i in range(3):
        wi = w[:, i] - geom.origin[i]
        g = np.floor((wi / geom.s) * float(2 ** BITS))
        G[:, i] = np.clip(g, 0, geom.M[i] * 2 ** BITS - 1).astype(np.int64)
    return G


def wrap_and_quantize(points, geom):
    """wrap() then quantize() (no images)."""
    w = wrap(points, geom)
    return w, quantize(w, geom)


class Box:
    __slots__ = ("level", "ix", "children", "parent", "pts", "id")

    def __init__(self, level, ix, parent, pts):
        self.level = level
        self.ix = tuple(int(v) for v in ix)
        self.children = []
        self.parent = parent
        self.pts = pts
        self.id = -1

    @property
    def is_leaf(self):
        return len(self.children) == 0

    def split(self, G):
        sh = BITS - self.level - 1
        for oz, oy, ox in itertools.product((0, 1), repeat=3):
            o = (ox, oy, oz)
            cix = tuple(2 * self.ix[i] + o[i] for i in range(3))
            if len(self.pts):
                sel = np.ones(len(self.pts), dtype=bool)
                for i in range(3):
                    sel &= ((G[self.pts, i] >> sh) & 1) == o[i]
                cp = self.pts[sel]
            else:
                cp = self.pts
            self.children.append(Box(self.level + 1, cix, self, cp))


class Forest:
    """Forest over the tiled domain; boxes carry integer indices on the global level grid."""

    def __init__(self, geom, G, n_s):
        self.geom = geom
        self.G = G
        self.n_s = n_s
        self.roots = []
        N = G.shape[0]
        allpts = np.arange(N)
        for m3 in range(geom.M[2]):
            for m2 in range(geom.M[1]):
                for m1 in range(geom.M[0]):
                    m = (m1, m2, m3)
                    sel = np.ones(N, dtype=bool)
                    for i in range(3):
                        sel &= (G[:, i] >> BITS) == m[i]
                    self.roots.append(Box(0, m, None, allpts[sel]))
        # (i) refine while a box holds more than n_s points (Sec. 3.1.1)
        stack = list(self.roots)
        while stack:
            b = stack.pop()
            if len(b.pts) > n_s and b.level < BITS:
                b.split(G)
                stack.extend(b.children)
        # (ii) 2:1 balance by fix-point iteration over the leaves (Sec. 3.1.1, 4.1.3)
        self._balance()
        self._index()

    def boxes(self):
        out = []
        stack = list(reversed(self.roots))
        while stack:
            b = stack.pop()
            out.append(b)
            stack.extend(reversed(b.children))
        return out

    def leaves(self):
        return [b for b in self.boxes() if b.is_leaf]

    def _balance(self):
        geom = self.geom
        ntot = np.array([geom.M[i] * 2 ** BITS for i in range(3)], dtype=np.int64)
        shifts = [s for s in itertools.product((-1, 0, 1), repeat=3)
                  if all(s[i] == 0 or geom.fperiodic[i] for i in range(3))]
        while True:
            leaves = self.leaves()
            lev = np.array([b.level for b in leaves])
            lo = np.array([[b.ix[i] << (BITS - b.level) for i in range(3)] for b in leaves], dtype=np.int64)
            hi = np.array([[(b.ix[i] + 1) << (BITS - b.level) for i in range(3)] for b in leaves], dtype=np.int64)
            to_split = []
            for a in range(len(leaves)):
                finer = lev >= lev[a] + 2
                if not np.any(finer):
                    continue
                touch = np.zeros(len(leaves), dtype=bool)
                for s in shifts:
                    off = np.array(s, dtype=np.int64) * ntot
                    ok = np.ones(len(leaves), dtype=bool)
                    for i in range(3):
                        # closed intervals [lo, hi] share a point
                        ok &= (lo[:, i] + off[i] <= hi[a, i]) & (lo[a, i] <= hi[:, i] + off[i])
                    touch |= ok
                if np.any(touch & finer):
                    to_split.append(leaves[a])
            if not to_split:
                return
            for b in to_split:
                b.split(self.G)

    def _index(self):
        allb = self.boxes()
        allb.sort(key=lambda b: b.level)
        for i, b in enumerate(allb):
            b.id = i
        self.by_id = allb
        self.nlevels = max(b.level for b in allb) + 1

    # ---- colleagues and the interaction recursion ------------------------------
    def _adjacent(self, a, b, shift):
        """Same-level boxes a and (b shifted by whole periods `shift`) share a boundary point."""
        for i in range(3):
            n = self.geom.M[i] * 2 ** a.level
            if abs(a.ix[i] - (b.ix[i] + shift[i] * n)) > 1:
                return False
        return True

    def interactions(self):
        """Run the telescoping recursion from all colleague pairs of root cubes.

        Returns (pw, direct):
          pw[l]   list of (target box, source box, shift) with both boxes non-leaf at level l;
          direct  list of (target box, source box, shift, l): K_R(nu_l) from every point
                  below the source box to every target in the leaves below the target box.
        `shift` counts whole periods per axis (0 on free axes); the source image sits at
        x_s + shift * L.
        """
        geom = self.geom
        shifts = [s for s in itertools.product((-1, 0, 1), repeat=3)
                  if all(s[i] == 0 or geom.fperiodic[i] for i in range(3))]
        pw = [[] for _ in range(self.nlevels)]
        direct = []

        def rec(A, S, sh, l):
            if not A.is_leaf and not S.is_leaf:
                pw[l].append((A, S, sh))
                for a in A.children:
                    for b in S.children:
                        if self._adjacent(a, b, sh):
                            rec(a, b, sh, l + 1)
            else:
                direct.append((A, S, sh, l))

        for A in self.roots:
            for S in self.roots:
                for sh in shifts:
                    if self._adjacent(A, S, sh):
                        rec(A, S, sh, 0)
        return pw, direct

    def leaves_below(self, b):
        if b.is_leaf:
            return [b]
        out = []
        for c in b.children:
            out.extend(self.leaves_below(c))
        return out
