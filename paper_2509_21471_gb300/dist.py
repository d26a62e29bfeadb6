"""One process per GPU (torchrun).

Weak scaling over independent systems: the near-field pass of one system has
no exchange step when every rank holds a whole system, so the ranks share no
data: rank r evaluates its own seeded system (seed index offset by 100 r).  The
only collectives are a barrier around the timed region and the maximum of the
elapsed times over ranks; the whole-job rate is (ranks x units per rank x
steps) / that maximum.

One system over several ranks: every rank builds the tree from all coordinates;
the target leaves are split into contiguous Morton ranges of about equal issued
pairs (dmk_stokes_partition_leaves), each rank owns its range's points and
their densities, and before the pass it receives the densities of its halo, the
points of the near-list leaves outside its range (dmk_stokes_halo_leaves):
halo_exchange below, one batch of point-to-point sends and receives.
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


def halo_exchange(values, owner, halo_points):
    """Fills values[halo_points] (rows of a [N, ...] tensor on this rank's
    device) from the ranks that own them, in one batch of point-to-point
    sends and receives.  owner[i] is the rank owning point i (every rank
    computes it from the partition); each rank sends the rows it owns that a
    peer's halo lists, in that peer's halo order.  Returns values."""
    import numpy as np
    world, me = dist.get_world_size(), dist.get_rank()
    halo_points = np.asarray(halo_points, dtype=np.int64)
    needs = [None] * world
    dist.all_gather_object(needs, halo_points.tolist())
    ops, recvs = [], []
    for q in range(world):
        if q == me:
            continue
        want = np.asarray(needs[q], dtype=np.int64)
        send_idx = want[owner[want] == me] if len(want) else want
        if len(send_idx):
            ops.append(dist.P2POp(dist.isend, values[torch.as_tensor(send_idx, device=values.device)].contiguous(), q))
        recv_idx = halo_points[owner[halo_points] == q] if len(halo_points) else halo_points
        if len(recv_idx):
            buf = torch.empty((len(recv_idx),) + tuple(values.shape[1:]), dtype=values.dtype, device=values.device)
            ops.append(dist.P2POp(dist.irecv, buf, q))
            recvs.append((recv_idx, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for idx, buf in recvs:
        values[torch.as_tensor(idx, device=values.device)] = buf
    return values
