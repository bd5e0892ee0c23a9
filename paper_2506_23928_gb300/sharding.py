"""Trajectories over ranks: one process per GPU, each advancing its own block of trajectories.

Trajectories are independent (the ensemble of Eq. 3 is an average over them), so the data
path has no collective: rank r of R takes the contiguous global ids of `shard`, and every
random draw is keyed by the global id, so a trajectory's path does not depend on R.  The
only exchange is host-side, at measurement times: the per-trajectory moments are gathered
and combined into the ensemble moments M, C and xi^2 (otvmc_ensemble), and a timing is
reduced to its maximum over ranks.
"""
import ctypes

import numpy as np

from . import abi


def shard(ntraj_total, rank, world):
    """(traj0, count) of rank `rank`: contiguous blocks, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or ntraj_total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(ntraj_total, world)
    count = base + (1 if rank < extra else 0)
    traj0 = rank * base + min(rank, extra)
    return traj0, count


def gather_moments(moments_local, ntraj_total, group=None):
    """All ranks' per-trajectory moments [n_meas][count_r][9] -> [n_meas][ntraj_total][9]
    in global trajectory order (every rank receives the whole array)."""
    import torch
    import torch.distributed as dist
    m = torch.as_tensor(np.ascontiguousarray(moments_local, dtype=np.float64))
    world = dist.get_world_size(group)
    counts = [shard(ntraj_total, r, world)[1] for r in range(world)]
    width = max(counts)
    n_meas = m.shape[0]
    pad = torch.zeros((n_meas, width, abi.OTVMC_MOMENTS), dtype=torch.float64)
    pad[:, :m.shape[1]] = m
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return np.concatenate([parts[r][:, :counts[r]].numpy() for r in range(world)], axis=1)


def ensemble(moments, n_sites):
    """Ensemble moments of one measurement time from per-trajectory moments [ntraj][9]:
    M[3], C[3][3], xi^2, standard error of M (otvmc_ensemble)."""
    mom = np.ascontiguousarray(moments, dtype=np.float64)
    M, C, dM = np.zeros(3), np.zeros((3, 3)), np.zeros(3)
    xi2 = ctypes.c_double()
    abi.check(abi.otvmc_ensemble(mom, mom.shape[0], n_sites, M, C, xi2, dM))
    return M, C, xi2.value, dM


def max_over_ranks(value, group=None):
    """Maximum of a host float over ranks (the step time of the slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
