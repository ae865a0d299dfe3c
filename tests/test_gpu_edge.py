"""Edge cases of the CUDA path against the oracle, element by element, through the C ABI.

* Pairs at the edge of the residual kernel's support, r = nu (1 -+ 1e-3): a uniform tree of
  one point per level-3 leaf (nu_3 = 1/8) with the points of neighbouring leaves 1/8 -+ 1.25e-4
  apart along every axis; the mixed path's half-precision pre-test must keep the pairs just
  inside and its FP32 test drop those just outside (Sec. 2.4, K_R vanishes for r >= nu).
* Periodic coordinates given exactly at L_i, below 0 and several periods away: wrapped into
  [0, L_i) (Eq. periodic-images) to the same result as the pre-wrapped input.
* More than n_s coincident points: the box is refined to the depth cap (18 levels) and kept as
  a leaf holding them all (reading of the depth cap); pairs at r = 0 are dropped.
* N = 1 and N < n_s (a single leaf).
* Every error the evaluation itself returns: non-neutral Laplace charges for D = 1, 2
  (Sec. 5.2), a free coordinate outside [0, L_i), a non-finite coordinate.
Bars: 1e-10 (plain FP64 path) and 1e-5 (mixed path), relative l2 over all targets and
components, as in test_gpu_parity.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dmk import evaluate
from paper_2606_27134_b300 import dmk, workloads as W

pytestmark = pytest.mark.gpu

BARS = {"fp64": 1e-10, "mixed": 1e-5}


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gpu(kernel, D, L, tol, x, rho, prec, n_s):
    plan = dmk.Plan(kernel, D, L, tol, precision=prec, n_s=n_s)
    u, g = plan.eval(torch.tensor(x, dtype=torch.float64, device="cuda"),
                     torch.tensor(rho, dtype=torch.float64, device="cuda"), grad=True)
    torch.cuda.synchronize()
    st = plan.stats()
    plan.close()
    return u.cpu().numpy(), g.cpu().numpy(), st


def support_edge_lattice():
    """8^3 points, one per level-3 leaf of the unit cube; neighbours along an axis alternate
    between 1/8 (1 - 1e-3) and 1/8 (1 + 1e-3) apart (also across the periodic boundary)."""
    n, nu = 8, 1.0 / 8
    d = 1e-3 * nu / 2
    c = (np.arange(n) + 0.5) * nu + np.where(np.arange(n) % 2 == 0, d, -d)
    x = np.stack(np.meshgrid(c, c, c, indexing="ij"), axis=-1).reshape(-1, 3)
    return x


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pairs_at_support_edge(prec):
    x = support_edge_lattice()
    N = x.shape[0]
    q = W.neutral_charges(N, 401).reshape(N, 1)
    ref = evaluate("laplace", 3, [1, 1, 1], 1e-6, x, q, n_s=1, grad=True)
    u, g, st = gpu("laplace", 3, [1, 1, 1], 1e-6, x, q, prec, 1)
    assert st["n_levels"] == ref.forest.nlevels == 4 and st["n_boxes"] == len(ref.forest.by_id)
    assert rel(u, ref.u) <= BARS[prec], rel(u, ref.u)
    assert rel(g, ref.grad) <= BARS[prec], rel(g, ref.grad)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_periodic_wrap_of_far_coordinates(prec):
    L, D, N = [1.0, 2.0, 0.5], 2, 600
    x = W.mixed_points(N, L, 402, D=D)
    rho = W.stokes_strengths("stokeslet", N, 403)
    xx = x.copy()
    xx[0, 0] = L[0]                         # exactly L_1 (wraps to 0)
    xx[1, 1] = L[1]                         # exactly L_2
    xx[2, 0] = -0.3                         # below 0
    xx[3, 1] = -3 * L[1] + 0.25             # three periods below
    xx[4, 0] = 5 * L[0] + 0.125             # five periods above
    xx[5, :2] = [-7 * L[0] + 0.5, 4 * L[1] + 1.0]
    ref = evaluate("stokeslet", D, L, 1e-6, xx, rho, n_s=40, grad=True)
    u, g, _ = gpu("stokeslet", D, L, 1e-6, xx, rho, prec, 40)
    assert rel(u, ref.u) <= BARS[prec] and rel(g, ref.grad) <= BARS[prec]
    # the same problem with the coordinates wrapped by hand
    w = xx.copy()
    for a in range(D):
        w[:, a] = np.mod(w[:, a], L[a])
        w[:, a] = np.where(w[:, a] >= L[a], 0.0, w[:, a])
    u2, g2, _ = gpu("stokeslet", D, L, 1e-6, w, rho, prec, 40)
    assert rel(u2, u) <= 1e-13 and rel(g2, g) <= 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_coincident_points_beyond_leaf_capacity(prec):
    L, N0, k, n_s = [1.0, 1.0, 1.0], 700, 300, 250
    x = W.uniform_points(N0, L, 404)
    x = np.vstack([x, np.tile([[0.3137, 0.6021, 0.4444]], (k, 1))])
    q = W.neutral_charges(N0 + k, 405).reshape(-1, 1)
    ref = evaluate("laplace", 3, L, 1e-6, x, q, n_s=n_s, grad=True)
    u, g, st = gpu("laplace", 3, L, 1e-6, x, q, prec, n_s)
    assert st["n_levels"] == ref.forest.nlevels == 19
    assert st["n_boxes"] == len(ref.forest.by_id)
    assert st["n_capped_leaves"] == 1
    assert rel(u, ref.u) <= BARS[prec]
    # gradients at the bars away from the stack of coincident points
    assert rel(g[:N0], ref.grad[:N0]) <= BARS[prec]
    # At the stack the field is the sum of the smooth parts of the 300 coincident charges over
    # 18 levels, O(max|u|), represented by a degree-p Chebyshev expansion on a box of side
    # h = 2^-18.  The expansion's derivative turns a coefficient rounding of eps max|u| into a
    # gradient error of about eps max|u| p^2 / (h / 2): that conditioning, not the bars of the
    # method, bounds the agreement there (eps = 2^-52 FP64 path, 2^-23 mixed path; p = 20).
    eps = 2.0 ** -52 if prec == "fp64" else 2.0 ** -23
    bound = 10 * eps * np.max(np.abs(ref.u)) * 20 ** 2 / (2.0 ** -18 / 2)
    assert np.max(np.abs(g[N0:] - ref.grad[N0:])) <= bound


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [("laplace", 3, [1, 1, 1], 1, 250), ("rotlet", 1, [2, 1, 1], 1, 250),
                                  ("laplace", 2, [1, 1, 0.5], 100, 250), ("stokeslet", 0, [1, 1, 1], 100, 250)],
                         ids=["laplace-3P-N1", "rotlet-1P-N1", "laplace-2P-N100", "stokeslet-0P-N100"])
def test_tiny_problems(case, prec):
    kernel, D, L, N, n_s = case
    x = W.uniform_points(N, L, 406)
    if kernel == "laplace":
        rho = (np.array([[0.7]]) if N == 1 else W.neutral_charges(N, 407).reshape(N, 1))
    else:
        rho = W.stokes_strengths(kernel, N, 407) if N > 1 else np.array([[0.3, -0.5, 0.9]])
    ref = evaluate(kernel, D, L, 1e-6, x, rho, n_s=n_s, grad=True)
    u, g, st = gpu(kernel, D, L, 1e-6, x, rho, prec, n_s)
    assert st["n_boxes"] == len(ref.forest.by_id)
    # a lone point's own images can give a zero field (or gradient) by symmetry, so the error
    # is measured against max(|reference|, the kernel's scale at the cube side s)
    s = min(L[:D]) if D > 0 else max(L)
    scale = np.linalg.norm(rho) / (4 * np.pi)
    for a, b, fl in ((u, ref.u, scale / s), (g, ref.grad, scale / s ** 2)):
        err = np.linalg.norm((a - b).ravel())
        assert err <= BARS[prec] * max(np.linalg.norm(b.ravel()), fl), (err, np.linalg.norm(b))


def _status(plan, x, rho):
    N = x.shape[0]
    dev = torch.device("cuda")
    xt = torch.tensor(x, dtype=torch.float64, device=dev)
    rt = torch.tensor(rho, dtype=torch.float64, device=dev).reshape(N, -1)
    u = torch.empty((N, plan.d_u), dtype=torch.float64, device=dev)
    lib = dmk.load()
    import ctypes
    return lib.dmk_eval(plan._h, N, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(rt.data_ptr()),
                        ctypes.c_void_p(u.data_ptr()), None), lib.dmk_last_error(plan._h).decode()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_evaluation_errors(prec):
    N = 300
    # Laplace, D = 2 and 1: net charge is refused (Sec. 5.2)
    for D, L in ((2, [1, 1, 0.5]), (1, [1, 1, 1])):
        plan = dmk.Plan("laplace", D, L, 1e-6, precision=prec, n_s=40)
        x = W.uniform_points(N, L, 408)
        q = W.neutral_charges(N, 409) + 0.01
        st, msg = _status(plan, x, q)
        assert st == 3 and "net charge" in msg
        st, _ = _status(plan, x, q - q.mean())
        assert st == 0
        plan.close()
    # free coordinate outside [0, L_i): above, below, exactly L_i
    plan = dmk.Plan("laplace", 2, [1, 1, 0.5], 1e-6, precision=prec, n_s=40)
    x = W.uniform_points(N, [1, 1, 0.5], 410)
    q = W.neutral_charges(N, 411)
    for bad in (0.5, -1e-9, 0.75):
        xb = x.copy()
        xb[17, 2] = bad
        st, msg = _status(plan, xb, q)
        assert st == 2 and "outside" in msg
    # non-finite coordinates, periodic or free
    for a, bad in ((0, np.nan), (1, np.inf), (2, -np.inf)):
        xb = x.copy()
        xb[5, a] = bad
        st, msg = _status(plan, xb, q)
        assert st == 2 and "non-finite" in msg
    # the plan stays usable after every error
    st, _ = _status(plan, x, q)
    assert st == 0
    plan.close()


@pytest.mark.parametrize("kernel,D,L", [("laplace", 2, [1.0, 1.0, 0.25]), ("rotlet", 3, [1.0, 1.0, 4.0])])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_pair_overlap_is_bitwise_neutral(kernel, D, L, precision):
    """The residual sums beside the far field (default) and in order give the same bits."""
    N = 20000
    x = torch.tensor(W.uniform_points(N, L, 611), device="cuda")
    q = torch.tensor(W.stokes_strengths(kernel, N, 612), device="cuda")
    p = dmk.Plan(kernel, D, L, 1e-6, precision=precision, n_s=100)
    u1, g1 = p.eval(x, q, grad=True)
    p.set_pair_overlap(False)
    u2, g2 = p.eval(x, q, grad=True)
    p.set_pair_overlap(True, 2)
    u3, g3 = p.eval(x, q, grad=True)
    assert torch.equal(u1, u2) and torch.equal(g1, g2)
    assert torch.equal(u1, u3) and torch.equal(g1, g3)
    p.close()
