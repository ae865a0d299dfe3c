"""Cube sharding (paper_2606_27134_b300/shard.py): partition, ghost cubes and the point exchange,
with two gloo ranks on the CPU, and the whole split evaluation with the oracle as each rank's
evaluator (its structure-factor hook completed by a gloo all-reduce): the union of the ranks'
results must equal one evaluation of all the points."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist
import torch.multiprocessing as mp

from oracle.dmk import evaluate
from oracle.params import Geometry
from oracle.tree import quantize, wrap, BITS
from paper_2606_27134_b300 import shard, workloads as W


def test_point_cubes_match_the_quantisation():
    for D, L in ((3, [1, 1, 6]), (2, [2, 1, 0.7]), (1, [3, 1, 1])):
        x = W.uniform_points(500, L, 7) + np.array([1.5, -2.25, 0.0]) * (np.arange(3) < D) * np.array(L)
        g = Geometry(D, L)
        G = quantize(wrap(x, g), g) >> BITS
        want = G[:, 0] + g.M[0] * (G[:, 1] + g.M[1] * G[:, 2])
        assert np.array_equal(shard.point_cubes(x, D, L), want)


def test_partition_is_contiguous_and_balanced():
    rng = np.random.default_rng(3)
    for n, world in ((16, 2), (16, 8), (27, 4), (5, 5), (64, 3)):
        w = rng.integers(1, 100, n)
        own = shard.partition_cubes(w, world)
        assert own[0] == 0 and own[-1] == world - 1
        assert np.all(np.diff(own) >= 0) and np.all(np.diff(own) <= 1)     # contiguous ranges
        loads = np.bincount(own, weights=w, minlength=world)
        assert loads.max() <= w.sum() / world + w.max()


def test_neighbours_by_brute_force():
    for M, per in (([1, 1, 6], [True] * 3), ([4, 3, 2], [True, False, False]), ([2, 2, 1], [True, True, True])):
        n = M[0] * M[1] * M[2]
        for m in range(n):
            a = np.array([m % M[0], (m // M[0]) % M[1], m // (M[0] * M[1])])
            want = set()
            for j in range(n):
                b = np.array([j % M[0], (j // M[0]) % M[1], j // (M[0] * M[1])])
                if j == m:
                    continue
                ok = True
                for i in range(3):
                    d = abs(int(a[i]) - int(b[i]))
                    if per[i]:
                        d = min(d, M[i] - d)
                    ok &= d <= 1
                if ok:
                    want.add(j)
            assert shard.neighbour_cubes(m, M, per) == want


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASE = dict(kernel="laplace", D=3, L=[1, 1, 6], tol=1e-6, N=900, n_s=40)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = CASE
        x = W.uniform_points(c["N"], c["L"], 61)
        q = W.neutral_charges(c["N"], 62).reshape(-1, 1)
        ids = np.arange(c["N"])
        cubes = shard.point_cubes(x, c["D"], c["L"])
        s, M, per = shard.tiling(c["D"], c["L"])
        owner = shard.partition_cubes(np.bincount(cubes, minlength=M[0] * M[1] * M[2]), world)
        ghosts = [shard.ghost_cubes(owner, M, per, r) for r in range(world)]
        # every rank starts with an arbitrary half of the points
        mine0 = (np.random.default_rng(5).random(c["N"]) < 0.5) == (rank == 0)
        ox, oq, oid, gx, gq = shard.route(x[mine0], q[mine0], ids[mine0], cubes[mine0], owner, ghosts, rank, world,
                                          tdist)
        # what each rank must hold: its cubes' points, and its ghost cubes' points
        assert np.array_equal(oid, np.nonzero(owner[cubes] == rank)[0])
        assert len(gx) == int(np.isin(cubes, ghosts[rank]).sum())
        own_cubes = np.nonzero(owner == rank)[0]

        def red(chi):
            t = torch.from_numpy(np.ascontiguousarray(np.stack([chi.real, chi.imag])))
            tdist.all_reduce(t)
            return t[0].numpy() + 1j * t[1].numpy()

        lx = np.vstack([ox, gx])
        lq = np.vstack([oq, gq])
        r = evaluate(c["kernel"], c["D"], c["L"], c["tol"], lx, lq, n_s=c["n_s"], grad=True, owned_cubes=own_cubes,
                     chi_reduce=red, targets=np.arange(len(ox)))
        out[rank] = (oid, r.u[:len(ox)].copy(), r.grad[:len(ox)].copy())
    finally:
        tdist.destroy_process_group()


def test_split_evaluation_with_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    c = CASE
    x = W.uniform_points(c["N"], c["L"], 61)
    q = W.neutral_charges(c["N"], 62).reshape(-1, 1)
    full = evaluate(c["kernel"], c["D"], c["L"], c["tol"], x, q, n_s=c["n_s"], grad=True)
    u = np.full_like(full.u, np.nan)
    g = np.full_like(full.grad, np.nan)
    for r in range(world):
        oid, ur, gr = out[r]
        u[oid] = ur
        g[oid] = gr
    assert np.isfinite(u).all()
    assert np.linalg.norm(u - full.u) <= 1e-13 * np.linalg.norm(full.u)
    assert np.linalg.norm(g - full.grad) <= 1e-13 * np.linalg.norm(full.grad)
