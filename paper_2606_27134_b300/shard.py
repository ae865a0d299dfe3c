"""One evaluation split over the ranks of a process group by cubes (host logic; spatial sharding).

The structure factor of Sec. 4.3 (Eq. structurefac) is a sum over the cubes of the tiling, and
a target's near field -- plane waves and residual sums (Sec. 3.1.4-3.1.5) -- reaches only the
cubes adjacent to its own.  So the evaluation shards by cubes:

* partition: each rank owns a contiguous range of cube indices m1 + M1 (m2 + M2 m3), balanced by
  the number of points in the cubes;
* ghosts: each rank also receives every point of the cubes adjacent to its own (the 26
  neighbours, wrapped along the exactly tiled periodic axes) that it does not own;
* each rank evaluates its own points with dmk_eval_shard from its own and its ghost points; the
  partial structure factors of the ranks are summed by one all-reduce inside the call.

The point exchange is one all-to-all; the structure factor all-reduce runs on the host through
the plan's pinned staging buffer (a few kB to a few MB).  The cube of a point is computed here
with the library's own sequence of rounded FP64 operations, so both sides agree on it.
"""
import ctypes

import numpy as np

KBITS = 18


def _wrap_axis(x, L):
    """x wrapped into [0, L): x - L floor(x / L); >= L -> - L; < 0 -> 0 (the library's order)."""
    v = x - L * np.floor(x / L)
    v = np.where(v >= L, v - L, v)
    return np.where(v < 0, 0.0, v)


def tiling(D, L):
    """(s, M, periodic) of the cube tiling of an exactly tiled cell (Sec. 4.1.1)."""
    L = [float(v) for v in L]
    s = min(L[:D]) if D > 0 else max(L)
    M, per = [], []
    for i in range(3):
        r = L[i] / s
        if i < D:
            m = int(round(r))
            if abs(r - m) > 1e-12 * max(1.0, r):
                raise NotImplementedError("sharding needs an exact tiling")
            M.append(m)
            per.append(True)
        else:
            M.append(max(1, int(np.ceil(r * (1 - 1e-12)))))
            per.append(False)
    return s, M, per


def point_cubes(points, D, L):
    """Cube index m1 + M1 (m2 + M2 m3) of every point (N, 3)."""
    s, M, per = tiling(D, L)
    x = np.asarray(points, dtype=np.float64)
    cube = np.zeros(x.shape[0], dtype=np.int64)
    stride = 1
    for i in range(3):
        v = _wrap_axis(x[:, i], float(L[i])) if per[i] else x[:, i]
        g = np.floor((v / s) * float(2 ** KBITS))
        g = np.clip(g, 0, M[i] * 2 ** KBITS - 1).astype(np.int64)
        cube += (g >> KBITS) * stride
        stride *= M[i]
    return cube


def partition_cubes(weights, world):
    """Owner rank of every cube: contiguous ranges of cube indices with balanced weights (every
    rank gets at least one cube when there are enough)."""
    w = np.asarray(weights, dtype=np.float64)
    n = len(w)
    owner = np.zeros(n, dtype=np.int64)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1] if cum[-1] > 0 else float(n)
    if cum[-1] <= 0:
        cum = np.arange(n + 1, dtype=np.float64)
    start = 0
    for r in range(world):
        # end of rank r: the first cube boundary at or beyond (r + 1)/world of the weight
        if r == world - 1:
            end = n
        else:
            end = int(np.searchsorted(cum, total * (r + 1) / world, side="left"))
            end = max(end, start + 1) if start < n else start
            end = min(end, n - (world - 1 - r)) if n - (world - 1 - r) > start else end
        owner[start:end] = r
        start = end
    return owner


def neighbour_cubes(m, M, periodic):
    """The cubes sharing a boundary point with cube m (26 at most), wrapped along periodic axes."""
    ix = [m % M[0], (m // M[0]) % M[1], m // (M[0] * M[1])]
    out = set()
    for d0 in (-1, 0, 1):
        for d1 in (-1, 0, 1):
            for d2 in (-1, 0, 1):
                if d0 == d1 == d2 == 0:
                    continue
                jx = []
                for i, d in enumerate((d0, d1, d2)):
                    v = ix[i] + d
                    if v < 0 or v >= M[i]:
                        if not periodic[i]:
                            break
                        v %= M[i]
                    jx.append(v)
                else:
                    j = jx[0] + M[0] * (jx[1] + M[1] * jx[2])
                    if j != m:
                        out.add(j)
    return out


def ghost_cubes(owner, M, periodic, rank):
    """Cubes adjacent to a cube of `rank` that `rank` does not own."""
    mine = np.nonzero(owner == rank)[0]
    g = set()
    for m in mine:
        g |= neighbour_cubes(int(m), M, periodic)
    return sorted(c for c in g if owner[c] != rank)


def route(points, strengths, ids, cubes, owner, ghosts, rank, world, dist):
    """Exchange points so that each rank holds its own points and its ghosts.

    points (n, 3), strengths (n, d), ids (n,) global point ids and cubes (n,) of the points this
    rank holds now (any distribution); owner: the owner rank of every cube; ghosts[r]: the ghost
    cubes of rank r.  Returns (own_points, own_strengths, own_ids, ghost_points, ghost_strengths).
    """
    import torch
    n, d = strengths.shape
    dests = []
    for r in range(world):
        send_own = owner[cubes] == r
        send_ghost = np.isin(cubes, np.asarray(ghosts[r], dtype=np.int64)) & ~send_own
        dests.append((np.nonzero(send_own)[0], np.nonzero(send_ghost)[0]))
    rec = 3 + d + 2                              # x, rho, id, flag (own = 1, ghost = 0)
    rows, counts = [], []
    for r in range(world):
        own_i, gh_i = dests[r]
        blk = np.zeros((len(own_i) + len(gh_i), rec))
        sel = np.concatenate([own_i, gh_i])
        blk[:, :3] = points[sel]
        blk[:, 3:3 + d] = strengths[sel]
        blk[:, 3 + d] = ids[sel]
        blk[:len(own_i), 4 + d] = 1.0
        rows.append(blk)
        counts.append(blk.shape[0])
    send = torch.from_numpy(np.vstack(rows) if rows else np.zeros((0, rec)))
    sc = torch.tensor(counts, dtype=torch.int64)
    rc = torch.zeros(world, dtype=torch.int64)
    dist.all_to_all_single(rc, sc)
    recv = torch.zeros((int(rc.sum()), rec), dtype=torch.float64)
    dist.all_to_all_single(recv, send, [int(v) for v in rc], counts)
    got = recv.numpy()
    own = got[:, 4 + d] == 1.0
    order = np.argsort(got[own, 3 + d], kind="stable")     # own points by global id
    og = got[own][order]
    gh = got[~own]
    gh = gh[np.argsort(gh[:, 3 + d], kind="stable")]
    return og[:, :3], og[:, 3:3 + d], og[:, 3 + d].astype(np.int64), gh[:, :3], gh[:, 3:3 + d]


def chi_allreduce(group):
    """A dmk_chi_reduce_fn that sums the host buffer over `group` (torch.distributed, any
    backend that reduces CPU tensors, e.g. gloo)."""
    import torch
    import torch.distributed as tdist
    from .dmk import CHI_REDUCE_FN

    def fn(ptr, n, ctx):
        try:
            arr = np.ctypeslib.as_array(ptr, shape=(int(n),))
            t = torch.from_numpy(arr)
            tdist.all_reduce(t, group=group)
            return 0
        except Exception:
            return 1
    return CHI_REDUCE_FN(fn)


def eval_shard(plan, own_points, own_strengths, ghost_points, ghost_strengths, cube_owned, reduce_fn, grad=False,
               device="cuda"):
    """dmk_eval_shard on this rank's own and ghost points (host numpy arrays in; torch CUDA
    results for the own points out)."""
    import torch
    from . import dmk
    lib = dmk.load()
    pts = np.vstack([np.asarray(own_points, dtype=np.float64).reshape(-1, 3),
                     np.asarray(ghost_points, dtype=np.float64).reshape(-1, 3)])
    rho = np.vstack([np.asarray(own_strengths, dtype=np.float64).reshape(-1, plan.d_rho),
                     np.asarray(ghost_strengths, dtype=np.float64).reshape(-1, plan.d_rho)])
    n_own = int(np.asarray(own_points).reshape(-1, 3).shape[0])
    N = pts.shape[0]
    xt = torch.tensor(pts, dtype=torch.float64, device=device)
    rt = torch.tensor(rho, dtype=torch.float64, device=device)
    u = torch.empty((max(n_own, 1), plan.d_u), dtype=torch.float64, device=device)
    g = torch.empty((max(n_own, 1), 3, plan.d_u), dtype=torch.float64, device=device) if grad else None
    owned = (ctypes.c_int * len(cube_owned))(*[int(v) for v in cube_owned])
    vp = ctypes.c_void_p
    st = lib.dmk_eval_shard(plan._h, N, n_own, vp(xt.data_ptr()), vp(rt.data_ptr()), vp(u.data_ptr()),
                            vp(g.data_ptr()) if grad else None, owned, reduce_fn, None)
    dmk._check(st, plan._h)
    return u[:n_own], (g[:n_own] if grad else None)
