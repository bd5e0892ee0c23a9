"""The linear stochastic Schroedinger equation (App. B) on the GPU: whole trajectories against the
oracle's linear otVMC (identical chains, parameters, and the normalisation ln Q at every
measured row), for the Jastrow, tied Jastrow and RBM ansaetze; and the Q-weighted ensemble
of the 8-spin workload against the exact Lindblad solution."""
import numpy as np
import pytest

from gpu_helpers import Case, require_gpu, to_dev_complex, from_dev_complex, unpack, rel_err, torch
import synth
from oracle import lindblad, trajectories as tr
from oracle.ansatz import RBM, lj_ansatz
from oracle.model import dense_hamiltonian, dense_jump_ops, coherent_x_state
from oracle.observables import ensemble_weighted, moments_from_rho
from paper_2506_23928_gb300 import abi
from paper_2506_23928_gb300.abi import check

pytestmark = pytest.mark.gpu
FP64, MIXED = abi.OTVMC_PREC_FP64, abi.OTVMC_PREC_MIXED


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _run(ans, P, n, T, ns, steps, dt, seed, precision, scheme, eps, theta0, every=1):
    desc = abi.RunDesc(ntraj=T, traj0=0, ns=ns, n_steps=steps, step0=0, n_sweep=2, dt=dt, scheme=scheme,
                       precision=precision, reg=abi.OTVMC_REG_SHIFT, eps=eps, snr_thresh=4.0, seed=seed,
                       measure_every=every, measure_final=1, use_graph=0)
    nm = abi.otvmc_run_n_meas(desc)
    theta = to_dev_complex(np.tile(theta0, (T, 1))).reshape(T, P, 2)
    spins = torch.zeros((T, ns, (n + 63) // 64), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(ans.handle, T, 0, ns, seed, spins))
    nb = abi.otvmc_run_workspace_bytes(ans.handle, desc)
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((nm, T, 9), dtype=torch.float64, device="cuda")
    lnq = torch.zeros(T, dtype=torch.float64, device="cuda")
    rows = torch.zeros((nm, T), dtype=torch.float64, device="cuda")
    check(abi.otvmc_run_trajectories_linear(ans.handle, desc, theta, spins, mom, lnq, rows, work, nb))
    return from_dev_complex(theta)[..., 0], unpack(spins, n), mom.cpu().numpy(), lnq.cpu().numpy(), rows.cpu().numpy()


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("kind,scheme", [("jastrow", abi.OTVMC_HEUN), ("jastrow", abi.OTVMC_MIDPOINT),
                                         ("lj", abi.OTVMC_HEUN), ("rbm", abi.OTVMC_MIDPOINT)])
def test_linear_run_matches_oracle(kind, scheme, precision):
    import paper_2506_23928_gb300 as pkg
    c = Case((7,), h=0.8, kappa=0.2, gamma=0.05)
    n = c.n
    if kind == "jastrow":
        ans, oans = c.ans, c.oans
    elif kind == "lj":
        ans, oans = pkg.Ansatz(c.model, kind=abi.OTVMC_LJ, d=1), lj_ansatz(n, 1)
    else:
        ans, oans = pkg.Ansatz(c.model, kind=abi.OTVMC_RBM, n_hidden=4), RBM(n, 4)
    P = ans.P
    assert P == oans.P
    T, ns, steps, dt, seed, eps = 2, 128, 3, 0.01, 515, 1e-3
    theta0 = synth.random_theta(3, 1, P, 0.1)[0]
    th, sig, mom, lnq, rows = _run(ans, P, n, T, ns, steps, dt, seed, precision, scheme, eps, theta0)
    sname = "heun" if scheme == abi.OTVMC_HEUN else "midpoint"
    lq = []
    oth, osig, om, oq = tr.run_mc(c.omodel, oans, T, ns, steps, dt, seed, sname, n_sweep=2, eps=eps,
                                  theta0=theta0, linear=True, lnq_out=lq)
    assert np.array_equal(sig, osig)
    tol = 1e-8 if precision == FP64 else 1e-4
    assert rel_err(th - theta0, oth - theta0) < tol
    # ln Q: twice the real part of the mean of v^lin per evaluation, so the mixed path's FP32
    # estimators carry into it at their own ~1e-5 level
    qtol = 1e-10 if precision == FP64 else 1e-5
    assert np.abs(rows - lq[0]).max() < qtol * max(1.0, np.abs(lq[0]).max())
    assert np.abs(lnq - lq[0][-1]).max() < qtol * max(1.0, np.abs(lq[0]).max())
    assert np.abs(lq[0][-1]).max() > 1e-4  # the norm moved
    want = np.concatenate([om, oq[..., [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]], axis=-1)
    assert rel_err(mom, want) < (1e-8 if precision == FP64 else 1e-5)


def test_linear_ensemble_matches_lindblad():
    """The 8-spin workload (h = 1, decay 0.1, Heun, dt = 0.01) on the linear SSE, 1024
    trajectories: the Q-weighted magnetisation (App. B) within 4 standard errors (+2e-3) of the
    exact Lindblad solution at t = 0.1, 0.2, 0.3, and the mean of Q within 4 standard errors of 1
    (the linear SSE preserves the trace on average)."""
    w = synth.WORKLOADS["chain8_jastrow"]
    c = Case(w.extent, alpha=w.alpha, h=w.h, kappa=w.kappa, gamma=w.gamma)
    T, steps, every = 1024, 30, 10
    _, _, mom, lnq, rows = _run(c.ans, c.P, c.n, T, w.ns, steps, w.dt, 13, MIXED, abi.OTVMC_HEUN, 1e-4,
                                np.zeros(c.P, complex), every=every)
    psi = coherent_x_state(w.n)
    _, recs = lindblad.evolve(np.outer(psi, psi.conj()), dense_hamiltonian(c.omodel), dense_jump_ops(c.omodel),
                              steps * w.dt, w.dt, observe=lambda r: moments_from_rho(r, w.n)[0], every=every)
    for i in range(1, mom.shape[0]):
        Q = np.exp(rows[i])
        q = np.zeros((T, 3, 3))
        M, _, dM = ensemble_weighted(mom[i, :, :3], q, Q)
        assert np.all(np.abs(M - recs[i]) <= 4 * dM + 2e-3), (i, M, recs[i], dM)
        assert abs(Q.mean() - 1.0) < 4 * Q.std(ddof=1) / np.sqrt(T) + 1e-3
