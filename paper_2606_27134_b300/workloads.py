"""Seeded synthetic inputs shaped like the paper's workloads.

Holds no arithmetic of the method: only random points and strengths.  Both the
CUDA path's tests and the oracle's tests draw their inputs from here.

* uniform points on [0,L1)x[0,L2)x[0,L3) (Sec. 6.2);
* "half uniform, half clustered near the centre of one top-level cube" (Tables 2
  and 6): the clustered half is Gaussian with sigma = 0.05 s around the centre of
  the first cube of side s = min periodic length (or max L for D = 0), wrapped;
* Gaussian clusters (sigma = 0.02) for an adaptive tree;
* the singly periodic pipe of Sec. 6 (Fig. cylinder_stokeslet): trapezoidal nodes on a cylinder
  around the periodic x1 axis, a fixed number of points per unit length;
* neutral +-1 charges, uniform charges minus their mean, N(0,1) vectors minus their
  mean, stresslet q (x) n with n uniform on the sphere, N(0,1) rotlet torques.
"""
import numpy as np


def _rng(seed):
    return np.random.default_rng(seed)


def uniform_points(N, L, seed):
    return _rng(seed).random((N, 3)) * np.asarray(L, dtype=np.float64)


def _wrap_into(x, L):
    L = np.asarray(L, dtype=np.float64)
    x = np.mod(x, L)
    return np.where(x >= L, 0.0, x)


def mixed_points(N, L, seed, D=None):
    """Half uniform, half N(centre of the first cube, (0.05 s)^2), wrapped into the cell."""
    rng = _rng(seed)
    L = np.asarray(L, dtype=np.float64)
    s = float(np.min(L)) if D is None else (float(np.min(L[:D])) if D > 0 else float(np.max(L)))
    n1 = N // 2
    a = rng.random((n1, 3)) * L
    centre = np.minimum(np.array([s / 2, s / 2, s / 2]), L / 2)
    b = centre + 0.05 * s * rng.standard_normal((N - n1, 3))
    return _wrap_into(np.vstack([a, b]), L)


def clustered_points(N, L, seed, n_centers=64, sigma=0.02):
    """N points from n_centers Gaussian clusters (centres uniform), wrapped periodically."""
    rng = _rng(seed)
    L = np.asarray(L, dtype=np.float64)
    centres = rng.random((n_centers, 3)) * L
    per = np.full(n_centers, N // n_centers)
    per[: N - per.sum()] += 1
    pts = np.vstack([c + sigma * rng.standard_normal((k, 3)) for c, k in zip(centres, per)])
    return _wrap_into(pts, L)


def cylinder_points(L1, per_unit=10000, n_theta=100, radius=0.4, centre=(0.5, 0.5)):
    """Trapezoidal nodes on the cylinder {(x1, c2 + r cos t, c3 + r sin t)} of the cell
    [0, L1) x [0, 1)^2: n_theta equispaced angles times per_unit / n_theta equispaced axial
    positions per unit of L1 (N = per_unit L1 points; the paper's pipe has 10,000 per unit
    length, its radius is not stated: 0.4 here)."""
    n_ax = int(round(L1 * per_unit / n_theta))
    x1 = (np.arange(n_ax) + 0.5) * (L1 / n_ax)
    t = 2 * np.pi * np.arange(n_theta) / n_theta
    X1, T = np.meshgrid(x1, t, indexing="ij")
    return np.stack([X1.ravel(), centre[0] + radius * np.cos(T.ravel()), centre[1] + radius * np.sin(T.ravel())], 1)


def neutral_charges(N, seed):
    """Random signs +-1 shifted to zero net charge."""
    s = _rng(seed).choice([-1.0, 1.0], N)
    return s - s.mean()


def balanced_charges(N, seed):
    """Exactly N/2 charges +1 and N/2 charges -1 (N even), randomly permuted."""
    q = np.ones(N)
    q[N // 2:] = -1.0
    return _rng(seed).permutation(q)


def uniform_charges(N, seed):
    """U[-1,1] minus the mean."""
    q = _rng(seed).uniform(-1.0, 1.0, N)
    return q - q.mean()


def stokes_strengths(kernel, N, seed):
    rng = _rng(seed)
    if kernel == "stokeslet":
        f = rng.standard_normal((N, 3))
        return f - f.mean(axis=0)
    if kernel == "stresslet":
        qv = rng.standard_normal((N, 3))
        n = rng.standard_normal((N, 3))
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        return (qv[:, :, None] * n[:, None, :]).reshape(N, 9)
    if kernel == "rotlet":
        return rng.standard_normal((N, 3))
    if kernel == "laplace":
        return neutral_charges(N, seed).reshape(N, 1)
    raise ValueError(kernel)
