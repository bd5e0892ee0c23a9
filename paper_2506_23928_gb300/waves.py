"""Trajectories admitted in waves by their device-memory footprint.

A batch of trajectories whose workspace does not fit the memory at hand is run as
consecutive waves on one GPU: each wave is a contiguous block of trajectory ids, sized so
that its workspace (`otvmc_run_workspace_bytes`) plus its own state (theta, chains, moments)
fits the given budget.  Every random draw is keyed by the global trajectory id, so a
trajectory's path does not depend on the wave it runs in: the waves give the results of one
batch.  One workspace, of the largest wave's size, is allocated once and reused.
"""
from . import abi
from .abi import check


def plan(ntraj, bytes_for, budget):
    """[(offset, count), ...] covering 0..ntraj-1 in order with the largest count c such that
    bytes_for(c) <= budget (bytes_for non-decreasing); raises MemoryError if one trajectory
    does not fit."""
    if ntraj <= 0:
        return []
    if bytes_for(1) > budget:
        raise MemoryError("one trajectory needs %d bytes, more than the budget of %d" % (bytes_for(1), budget))
    lo, hi = 1, ntraj
    while lo < hi:  # largest c with bytes_for(c) <= budget
        mid = (lo + hi + 1) // 2
        if bytes_for(mid) <= budget:
            lo = mid
        else:
            hi = mid - 1
    return [(k, min(lo, ntraj - k)) for k in range(0, ntraj, lo)]


def _state_bytes(P, ns, words, n_meas, count):
    return count * (P * 16 + ns * words * 8 + n_meas * abi.OTVMC_MOMENTS * 8)


def run(ansatz, desc, theta, spins, moments, budget, stream=None):
    """otvmc_run_trajectories over `desc.ntraj` trajectories in waves that fit `budget` bytes.

    theta [ntraj][P][2] float64, spins [ntraj][ns][words] int64 and moments [n_meas][ntraj][9]
    float64 are torch CUDA tensors of the whole batch (moments may be None when the descriptor
    measures nothing); they are updated in place.  Returns the wave plan."""
    import torch
    T = desc.ntraj
    P = theta.shape[1]
    words = spins.shape[2]
    n_meas = abi.otvmc_run_n_meas(desc)

    def sub(offset, count):
        d = abi.RunDesc(**{f: getattr(desc, f) for f, _ in abi.RunDesc._fields_})
        d.ntraj = count
        d.traj0 = desc.traj0 + offset
        return d

    def bytes_for(count):
        return abi.otvmc_run_workspace_bytes(ansatz, sub(0, count)) + _state_bytes(P, desc.ns, words, n_meas, count)

    waves = plan(T, bytes_for, budget)
    if not waves:
        return waves
    nb = max(abi.otvmc_run_workspace_bytes(ansatz, sub(o, c)) for o, c in waves)
    work = torch.zeros(nb, dtype=torch.uint8, device=theta.device)
    for o, c in waves:
        th = theta[o:o + c]
        sp = spins[o:o + c]
        mo = torch.zeros((n_meas, c, abi.OTVMC_MOMENTS), dtype=torch.float64, device=theta.device) if n_meas else None
        check(abi.otvmc_run_trajectories(ansatz, sub(o, c), th, sp, mo, work, nb, stream))
        if n_meas:
            moments[:, o:o + c] = mo
    return waves
