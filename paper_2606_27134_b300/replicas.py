"""Whole-job figures when every rank evaluates its own independent problem (replicas).

The evaluation does not shard across GPUs here: each rank runs a full dmk_eval on its own
points and no collective touches the data path.  The job's step is over when the slowest rank
is done, so the job step time is the maximum of the ranks' step times, and the job throughput
counts the targets of every rank over that time.  The only collective is this reduction of
timings, on whatever backend the process group uses (NCCL on GPUs, gloo in the CPU tests).
"""
import torch


def max_over_ranks(value, dist=None, device=None):
    """Maximum of a per-rank float over the process group (the value itself without one)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_local, step_ms, dist=None, device=None):
    """(targets/s of the whole job, job step time in ms) for n_local targets per rank."""
    world = dist.get_world_size() if dist is not None else 1
    t = max_over_ranks(step_ms, dist, device)
    return world * n_local / (t / 1e3), t
