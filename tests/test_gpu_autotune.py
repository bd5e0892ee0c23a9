"""Launch-shape autotuner (otvmc_autotune_run): it times the candidate shapes (sub-batches,
solver groups) of a batch, records the fastest, and leaves the caller's state untouched; runs
before and after the record give the same results bit for bit."""
import numpy as np
import pytest

from gpu_helpers import Case, require_gpu, torch
import synth
from paper_2506_23928_gb300 import abi
from paper_2506_23928_gb300.abi import check

pytestmark = pytest.mark.gpu
MIXED = abi.OTVMC_PREC_MIXED


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()
    yield
    abi.otvmc_autotune_clear()


def _desc(ntraj, ns, precision=MIXED):
    return abi.RunDesc(ntraj=ntraj, traj0=0, ns=ns, n_steps=3, step0=0, n_sweep=2, dt=0.01, scheme=abi.OTVMC_HEUN,
                       precision=precision, reg=abi.OTVMC_REG_SHIFT, eps=1e-3, snr_thresh=4.0, seed=7,
                       measure_every=1, measure_final=1, use_graph=0)


def _start(ans, P, n, d, theta0):
    theta = torch.from_numpy(np.tile(theta0, (d.ntraj, 1)).view(np.float64).copy()).cuda().reshape(d.ntraj, P, 2)
    spins = torch.zeros((d.ntraj, d.ns, (n + 63) // 64), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(ans.handle, d.ntraj, 0, d.ns, d.seed, spins))
    return theta, spins


def _run(ans, P, n, d, theta0):
    theta, spins = _start(ans, P, n, d, theta0)
    nb = abi.otvmc_run_workspace_bytes(ans.handle, d)
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((abi.otvmc_run_n_meas(d), d.ntraj, abi.OTVMC_MOMENTS), dtype=torch.float64, device="cuda")
    check(abi.otvmc_run_trajectories(ans.handle, d, theta, spins, mom, work, nb))
    return theta.cpu().numpy(), spins.cpu().numpy(), mom.cpu().numpy()


def _tune(ans, P, n, d, theta0):
    theta, spins = _start(ans, P, n, d, theta0)
    th0, sp0 = theta.clone(), spins.clone()
    nb = abi.otvmc_autotune_workspace_bytes(ans.handle, d)
    assert nb > abi.otvmc_run_workspace_bytes(ans.handle, d)
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    st, pipes, groups, ms = abi.otvmc_autotune_run(ans.handle, d, theta, spins, work, nb)
    check(st)
    assert torch.equal(theta, th0) and torch.equal(spins, sp0)
    assert abi.otvmc_autotune_run(ans.handle, d, theta, spins, work, nb - 256)[0] == abi.OTVMC_ERR_WORKSPACE
    return pipes, groups, ms


def test_autotuned_jastrow_batch_gives_the_same_results():
    """48 trajectories (candidates: 1, 2 or 4 sub-batches x solver groups 1, 2, 4 or the rule)."""
    c = Case((10,), kappa=0.1)
    d = _desc(48, 64)
    th0 = np.zeros(c.P, complex)
    before = _run(c.ans, c.P, c.n, d, th0)
    pipes, groups, ms = _tune(c.ans, c.P, c.n, d, th0)
    assert pipes in (1, 2, 4) and groups in (0, 1, 2, 4) and ms > 0
    after = _run(c.ans, c.P, c.n, d, th0)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


def test_autotuned_rbm_batch_gives_the_same_results():
    import paper_2506_23928_gb300 as pkg
    w = synth.WORKLOADS["chain8_jastrow"]
    c = Case(w.extent, alpha=w.alpha, h=w.h, kappa=w.kappa, gamma=w.gamma)
    rbm = pkg.Ansatz(c.model, kind=abi.OTVMC_RBM, n_hidden=16)
    th0 = np.zeros(rbm.P, complex)
    g = synth.rng(5)
    th0[c.n + 16:] = g.normal(0, 0.05, c.n * 16) + 1j * g.normal(0, 0.05, c.n * 16)
    d = _desc(16, 64)
    before = _run(rbm, rbm.P, c.n, d, th0)
    pipes, groups, ms = _tune(rbm, rbm.P, c.n, d, th0)
    assert pipes in (1, 2) and ms > 0
    after = _run(rbm, rbm.P, c.n, d, th0)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
