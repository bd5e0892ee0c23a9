"""Grouped runs (otvmc_run_trajectories_grouped): several batches of one ansatz with their own
sample counts in one call, each on its own forked stream.  Each group's theta, chains and
measured moments equal those of the same descriptor run by itself, bit for bit (the draws are
keyed by global trajectory id and step, and no group shares workspace with another)."""
import numpy as np
import pytest

from gpu_helpers import Case, require_gpu, torch
import synth
from paper_2506_23928_gb300 import abi

pytestmark = pytest.mark.gpu
MIXED = abi.OTVMC_PREC_MIXED


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _desc(ntraj, traj0, ns, steps=3, precision=MIXED, every=1, seed=5):
    return abi.RunDesc(ntraj=ntraj, traj0=traj0, ns=ns, n_steps=steps, step0=0, n_sweep=2, dt=0.01,
                       scheme=abi.OTVMC_HEUN, precision=precision, reg=abi.OTVMC_REG_SHIFT, eps=1e-3,
                       snr_thresh=4.0, seed=seed, measure_every=every, measure_final=1, use_graph=0)


def _state(ans, P, n, d, theta0):
    theta = torch.from_numpy(np.tile(theta0, (d.ntraj, 1)).view(np.float64).copy()).cuda().reshape(d.ntraj, P, 2)
    spins = torch.zeros((d.ntraj, d.ns, (n + 63) // 64), dtype=torch.int64, device="cuda")
    abi.check(abi.otvmc_init_chains(ans.handle, d.ntraj, d.traj0, d.ns, d.seed, spins))
    mom = torch.zeros((abi.otvmc_run_n_meas(d), d.ntraj, abi.OTVMC_MOMENTS), dtype=torch.float64, device="cuda")
    return theta, spins, mom


def _separate(ans, P, n, descs, theta0):
    out = []
    for d in descs:
        th, sp, mo = _state(ans, P, n, d, theta0)
        nb = abi.otvmc_run_workspace_bytes(ans.handle, d)
        work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        abi.check(abi.otvmc_run_trajectories(ans.handle, d, th, sp, mo, work, nb))
        out.append((th.cpu().numpy(), sp.cpu().numpy(), mo.cpu().numpy()))
    return out


def _grouped(ans, P, n, descs, theta0):
    st = [_state(ans, P, n, d, theta0) for d in descs]
    nb = abi.otvmc_run_grouped_workspace_bytes(ans.handle, descs)
    assert nb >= sum(abi.otvmc_run_workspace_bytes(ans.handle, d) for d in descs)
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    abi.check(abi.otvmc_run_trajectories_grouped(ans.handle, descs, [s[0] for s in st], [s[1] for s in st],
                                                 [s[2] for s in st], work, nb))
    return [(s[0].cpu().numpy(), s[1].cpu().numpy(), s[2].cpu().numpy()) for s in st]


def _rbm_case():
    import paper_2506_23928_gb300 as pkg
    w = synth.WORKLOADS["chain8_jastrow"]
    c = Case(w.extent, alpha=w.alpha, h=w.h, kappa=w.kappa, gamma=w.gamma)
    m = 16
    rbm = pkg.Ansatz(c.model, kind=abi.OTVMC_RBM, n_hidden=m)
    th0 = np.zeros(rbm.P, complex)
    g = synth.rng(3)
    th0[c.n + m:] = g.normal(0, 0.05, c.n * m) + 1j * g.normal(0, 0.05, c.n * m)
    return c, rbm, th0


def test_grouped_rbm_sample_counts_equal_separate_runs():
    """An RBM ensemble spread over three sample counts (N = 8, M = 16, P = 152: N_s = 64 and 128
    take the push-through T path, 256 the S path), as in a workload whose trajectories use
    several N_s: one grouped call equals the three calls, in every output bit."""
    c, rbm, th0 = _rbm_case()
    descs = [_desc(6, 0, 64), _desc(5, 6, 128), _desc(4, 11, 256)]
    sep = _separate(rbm, rbm.P, c.n, descs, th0)
    grp = _grouped(rbm, rbm.P, c.n, descs, th0)
    for a, b in zip(sep, grp):
        for k in range(3):
            assert np.array_equal(a[k], b[k])


def test_grouped_jastrow_with_pipelined_group_equals_separate_runs():
    """Jastrow (N = 10) groups of different size and N_s; the group of 40 trajectories runs as two
    forked sub-batches inside its own forked stream; a group with another precision and without
    measurements rides along.  Equal to the separate calls bit for bit."""
    c = Case((10,), kappa=0.1)
    th0 = np.zeros(c.P, complex)
    descs = [_desc(40, 0, 64), _desc(8, 40, 256), _desc(3, 48, 128, precision=abi.OTVMC_PREC_FP64, every=0)]
    sep = _separate(c.ans, c.P, c.n, descs, th0)
    grp = _grouped(c.ans, c.P, c.n, descs, th0)
    for a, b in zip(sep, grp):
        for k in range(3):
            assert np.array_equal(a[k], b[k])


def test_grouped_rejects_bad_arguments():
    c = Case((8,), kappa=0.1)
    d = _desc(2, 0, 64)
    th, sp, mo = _state(c.ans, c.P, c.n, d, np.zeros(c.P, complex))
    nb = abi.otvmc_run_grouped_workspace_bytes(c.ans.handle, [d])
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    assert abi.otvmc_run_grouped_workspace_bytes(c.ans.handle, [d] * (abi.OTVMC_MAX_GROUPS + 1)) == 0
    assert abi.otvmc_run_trajectories_grouped(c.ans.handle, [d], [th], [sp], [mo], work, nb - 256) == \
        abi.OTVMC_ERR_WORKSPACE
    assert abi.otvmc_run_trajectories_grouped(c.ans.handle, [d], [th], [sp], [None], work, nb) == abi.OTVMC_ERR_INVALID
    assert abi.otvmc_run_trajectories_grouped(c.ans.handle, [d], [th], [sp], [mo], work, nb) == abi.OTVMC_OK
