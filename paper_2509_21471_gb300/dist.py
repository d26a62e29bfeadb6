"""One process per GPU (torchrun): weak scaling over independent systems.

The near-field pass of one system has no exchange step when every rank holds a
whole system, so the ranks share no data: rank r evaluates its own seeded
system (seed index offset by 100 r).  The only collectives are a barrier
around the timed region and the maximum of the elapsed times over ranks; the
whole-job rate is (ranks x units per rank x steps) / that maximum.
"""
import os

import torch
import torch.distributed as dist

SEED_STRIDE = 100


def world_size():
    return int(os.environ.get("WORLD_SIZE", "1"))


def rank():
    return int(os.environ.get("RANK", "0"))


def init(backend=None):
    """Joins the process group when launched with more than one rank (NCCL with
    GPUs, gloo without)."""
    if world_size() > 1 and not dist.is_initialized():
        dist.init_process_group(backend or ("nccl" if torch.cuda.is_available() else "gloo"))


def finish():
    if dist.is_initialized():
        dist.destroy_process_group()


def barrier():
    if world_size() > 1:
        dist.barrier()


def max_over_ranks(v):
    """Maximum of a float over all ranks (every rank gets it)."""
    if world_size() == 1:
        return float(v)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def seed_index(base, r=None):
    """Seed index of this rank's system for a workload whose single-rank index is base."""
    return base + SEED_STRIDE * (rank() if r is None else r)


def job_rate(units_per_rank, steps, seconds_max):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world_size() * units_per_rank * steps / seconds_max
