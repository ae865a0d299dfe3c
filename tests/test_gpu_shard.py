"""dmk_eval_shard on the GPU: an evaluation split over cubes, the ranks emulated by host threads
on one GPU (each with its own plan and stream; they meet only in the host reduction of the
partial structure factors, never inside a kernel).  The union of the ranks' results must equal
the single evaluation of all points: to rounding against dmk_eval, and within the parity bars
against the oracle."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dmk import evaluate
from paper_2606_27134_b300 import dmk, shard, workloads as W

pytestmark = pytest.mark.gpu


def _barrier_reduce(world):
    """One dmk_chi_reduce_fn per emulated rank, summing through a shared host buffer."""
    bar = threading.Barrier(world, timeout=120)
    slots = [None] * world
    out = {}

    def make(rank):
        def fn(ptr, n, ctx):
            try:
                a = np.ctypeslib.as_array(ptr, shape=(int(n),))
                slots[rank] = a.copy()
                bar.wait()
                if rank == 0:
                    out["sum"] = np.sum(np.stack(slots), axis=0)
                bar.wait()
                a[:] = out["sum"]
                bar.wait()
                return 0
            except threading.BrokenBarrierError:
                return 1
        return dmk.CHI_REDUCE_FN(fn)
    return [make(r) for r in range(world)], bar


def run_sharded(kernel, D, L, tol, x, q, world, precision, n_s, owner=None, grad=True):
    cubes = shard.point_cubes(x, D, L)
    s, M, per = shard.tiling(D, L)
    nc = M[0] * M[1] * M[2]
    if owner is None:
        owner = shard.partition_cubes(np.bincount(cubes, minlength=nc), world)
    fns, bar = _barrier_reduce(world)
    plans = [dmk.Plan(kernel, D, L, tol, precision=precision, n_s=n_s) for _ in range(world)]
    res, errs = [None] * world, []

    def work(r):
        try:
            own = owner[cubes] == r
            gh = np.isin(cubes, shard.ghost_cubes(owner, M, per, r))
            u, g = shard.eval_shard(plans[r], x[own], q[own], x[gh], q[gh], (owner == r).astype(np.int32),
                                    fns[r], grad=grad)
            torch.cuda.synchronize()
            res[r] = (np.nonzero(own)[0], u.cpu().numpy(), None if g is None else g.cpu().numpy())
        except Exception as e:          # noqa: BLE001 -- reported below
            errs.append(e)
            bar.abort()

    th = [threading.Thread(target=work, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for p in plans:
        p.close()
    if errs:
        raise errs[0]
    du = res[0][1].shape[1]
    u = np.full((len(x), du), np.nan)
    g = np.full((len(x), 3, du), np.nan)
    for ids, ur, gr in res:
        u[ids] = ur
        if grad:
            g[ids] = gr
    return u, g, owner


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def whole(kernel, D, L, tol, x, q, precision, n_s):
    p = dmk.Plan(kernel, D, L, tol, precision=precision, n_s=n_s)
    u, g = p.eval(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"), grad=True)
    out = u.cpu().numpy(), g.cpu().numpy()
    p.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kernel,D,L,N,world", [
    ("laplace", 3, [1, 1, 6], 60000, 2),
    ("rotlet", 3, [1, 1, 16], 80000, 4),
    ("stokeslet", 1, [1, 1, 4], 40000, 3),
])
def test_shard_equals_whole(kernel, D, L, N, world, precision):
    x = W.uniform_points(N, L, 301)
    if kernel == "laplace":
        q = W.neutral_charges(N, 302).reshape(N, 1)
    elif precision == "fp64":
        # a net force / torque: the strength sums go through the reduction (the 1P Stokeslet
        # constant multiplies the total force)
        q = np.random.default_rng(302).standard_normal((N, 3)) + 0.25
    else:
        # forces summing to zero, as the Stokes workloads: with a net force the 1P velocity grows
        # logarithmically and its FP32 expansions lose relative precision in the gradient
        q = W.stokes_strengths("stokeslet", N, 302)
    u, g, owner = run_sharded(kernel, D, L, 1e-6, x, q, world, precision, 100)
    assert len(set(owner.tolist())) == world
    uw, gw = whole(kernel, D, L, 1e-6, x, q, precision, 100)
    assert np.isfinite(u).all() and np.isfinite(g).all()
    # summation order only: FP64 rounding on the plain path; on the mixed path the FP32 sums of
    # the two evaluations (different point orders within a leaf) each sit within the 1e-5 bar
    bar = 1e-12 if precision == "fp64" else 1e-5
    assert rel(u, uw) < bar and rel(g, gw) < bar


@pytest.mark.parametrize("kernel,D,L,N", [("laplace", 3, [1, 1, 6], 3000), ("stokeslet", 1, [1, 1, 4], 2000)])
def test_shard_matches_oracle(kernel, D, L, N):
    x = W.uniform_points(N, L, 311)
    if kernel == "laplace":
        q = W.neutral_charges(N, 312).reshape(N, 1)
    else:
        q = W.stokes_strengths("stokeslet", N, 312)
    u, g, _ = run_sharded(kernel, D, L, 1e-6, x, q, 2, "mixed", 40)
    ref = evaluate(kernel, D, L, 1e-6, x, q, n_s=40, grad=True)
    assert rel(u, ref.u) < 1e-5 and rel(g, ref.grad) < 1e-5


def test_rank_without_points():
    """Points only in cube 1 of six: the rank owning cubes 3-5 holds no point at all (no owned,
    no ghost), still takes part in the reduction, and the other rank's results are those of
    the whole evaluation."""
    L = [1, 1, 6]
    N = 4000
    x = W.uniform_points(N, [1, 1, 1], 321) + np.array([0, 0, 1.0])
    q = W.neutral_charges(N, 322).reshape(N, 1)
    owner = np.array([0, 0, 0, 1, 1, 1])
    u, g, _ = run_sharded("laplace", 3, L, 1e-6, x, q, 2, "fp64", 100, owner=owner)
    uw, gw = whole("laplace", 3, L, 1e-6, x, q, "fp64", 100)
    assert rel(u, uw) < 1e-12 and rel(g, gw) < 1e-12


def test_reduction_failure_is_reported():
    p = dmk.Plan("laplace", 3, [1, 1, 2], 1e-6, n_s=50)
    x = W.uniform_points(500, [1, 1, 2], 331)
    q = W.neutral_charges(500, 332).reshape(500, 1)
    fail = dmk.CHI_REDUCE_FN(lambda ptr, n, ctx: 1)
    with pytest.raises(dmk.DmkError, match="reduction"):
        shard.eval_shard(p, x, q, x[:0], q[:0], np.array([1, 1], dtype=np.int32), fail)
    # the plan stays usable
    u, _ = p.eval(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    assert torch.isfinite(u).all()
    p.close()
