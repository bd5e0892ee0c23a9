"""Trajectories in waves by device-memory footprint: the plan on the host (CPU), and on the
GPU that waves give the results of one batch (draws keyed by the global trajectory id)."""
import numpy as np
import pytest

from paper_2506_23928_gb300.waves import plan


def test_plan_covers_in_order_with_the_largest_fitting_wave():
    per = lambda c: 1000 + 300 * c  # noqa: E731
    for ntraj, budget in [(10, 4000), (7, 1300), (5, 10 ** 9), (1, 1300)]:
        waves = plan(ntraj, per, budget)
        assert [o for o, _ in waves] == list(range(0, ntraj, waves[0][1]))
        assert sum(c for _, c in waves) == ntraj
        size = waves[0][1]
        assert per(size) <= budget and (size == ntraj or per(size + 1) > budget)
    assert plan(0, per, 10) == []
    with pytest.raises(MemoryError):
        plan(3, per, 1200)


@pytest.mark.gpu
def test_waves_equal_one_batch():
    from gpu_helpers import Case, require_gpu, torch
    from paper_2506_23928_gb300 import abi, waves
    from paper_2506_23928_gb300.abi import check
    require_gpu()
    c = Case((8,), h=1.0, kappa=0.1, gamma=0.05)
    T, ns = 10, 256
    desc = abi.RunDesc(ntraj=T, traj0=3, ns=ns, n_steps=3, step0=0, n_sweep=2, dt=0.01, scheme=abi.OTVMC_MIDPOINT,
                       precision=abi.OTVMC_PREC_MIXED, reg=abi.OTVMC_REG_SHIFT, eps=1e-4, snr_thresh=4.0, seed=9,
                       measure_every=1, measure_final=1, use_graph=0)
    nm = abi.otvmc_run_n_meas(desc)

    def fresh():
        theta = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
        spins = torch.zeros((T, ns, c.W), dtype=torch.int64, device="cuda")
        check(abi.otvmc_init_chains(c.ans.handle, T, desc.traj0, ns, desc.seed, spins))
        return theta, spins, torch.zeros((nm, T, 9), dtype=torch.float64, device="cuda")

    th1, sp1, mo1 = fresh()
    nb = abi.otvmc_run_workspace_bytes(c.ans.handle, desc)
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    check(abi.otvmc_run_trajectories(c.ans.handle, desc, th1, sp1, mo1, work, nb))
    th2, sp2, mo2 = fresh()
    one = abi.RunDesc(**{f: getattr(desc, f) for f, _ in abi.RunDesc._fields_})
    one.ntraj = 1
    budget = 3 * abi.otvmc_run_workspace_bytes(c.ans.handle, one)  # about three trajectories a wave
    plan_ = waves.run(c.ans.handle, desc, th2, sp2, mo2, budget)
    assert len(plan_) >= 3
    assert torch.equal(th1, th2) and torch.equal(sp1, sp2) and torch.equal(mo1, mo2)
