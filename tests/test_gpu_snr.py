"""SNR-filtered eigen pseudo-inverse (otvmc_solve_snr) and whole trajectories with the SNR
regulariser, against the oracle's filter built on numpy's eigh, on the same samples."""
import numpy as np
import pytest

from gpu_helpers import Case, require_gpu, to_dev_complex, from_dev_complex, unpack, rel_err, torch
import synth
from oracle import tvmc, trajectories as tr
from paper_2506_23928_gb300 import abi
from paper_2506_23928_gb300.abi import check

pytestmark = pytest.mark.gpu
FP64, MIXED = abi.OTVMC_PREC_FP64, abi.OTVMC_PREC_MIXED


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _evaluate(c, T, ns, seed, scale, dt):
    th, _ = c.theta(seed, T, scale)
    sig, sp = c.spins(seed + 1, T, ns)
    dW = synth.random_normals(seed + 2, (T, c.nops), np.sqrt(dt))
    w = tvmc.mc_weights(ns)
    evs = [tvmc.evaluate(c.omodel, c.oans, th[t], sig[t], w, dW[t], dt) for t in range(T)]
    v = np.stack([tvmc.local_v(evs[t], dW[t], dt) for t in range(T)])
    return evs, v, sp, w


def _build(c, precision, T, ns, v, sp):
    P = c.P
    v_d = to_dev_complex(v)
    S = torch.zeros((T, P, P), dtype=torch.float64, device="cuda")
    G = torch.zeros((T, P, P), dtype=torch.float32, device="cuda") if precision == MIXED else None
    ob = torch.zeros((T, P), dtype=torch.float64, device="cuda")
    D = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, precision)
    check(abi.otvmc_build_S_F(c.ans.handle, None, sp, v_d, T, ns, precision, S, G, ob, D, work, nb))
    check(abi.otvmc_check(work))
    return S, ob, D, v_d


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,ns,thr", [(8, 1024, 4.0), (6, 304, 4.0), (9, 512, 40.0), (5, 200, 1e-9),
                                      (14, 512, 4.0), (24, 1024, 4.0), (31, 2048, 40.0), (20, 400, 1e-9),
                                      (32, 1024, 4.0)])
def test_solve_snr_matches_oracle(precision, n, ns, thr):
    """Odd and even P (Jacobi with and without the dummy index), a threshold that filters
    many modes, and a vanishing one (the plain pseudo-inverse); P = 105, 300, 496, 210 and 528
    take the tridiagonal path (Householder, implicit QL, one pass over the samples)."""
    c = Case((n,), h=0.8, kappa=0.1, gamma=0.05)
    T, dt = 3, 0.01
    evs, v, sp, w = _evaluate(c, T, ns, 61, 0.2, dt)
    S, ob, D, v_d = _build(c, precision, T, ns, v, sp)
    delta = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    lam = torch.zeros((T, c.P), dtype=torch.float64, device="cuda")
    nb = abi.otvmc_snr_workspace_bytes(c.ans.handle, T)
    assert nb == (256 if c.P <= 96 else 256 + 2 * T * c.P * c.P * 8 + 256)
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    check(abi.otvmc_solve_snr(c.ans.handle, T, ns, S, ob, sp, v_d, D, thr, 1e-12, delta, lam, work, nb))
    check(abi.otvmc_check(work))
    got = from_dev_complex(delta)[..., 0]
    for t in range(T):
        ev = evs[t]
        want = tvmc.solve_snr(ev["S"], ev["D"], ev["O"], v[t], w, snr_thresh=thr, eps_svd=1e-12)
        assert rel_err(got[t], want) < 1e-8
        assert rel_err(np.sort(lam[t].cpu().numpy()), np.linalg.eigvalsh(ev["S"].real)) < 1e-12


def test_solve_snr_rejects_what_it_does_not_hold():
    """P beyond the shared memory of one CTA (N = 80: P = 3240), a workspace without room for
    the decomposition, and the RBM."""
    import paper_2506_23928_gb300 as pkg
    T, ns = 1, 64
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    big = Case((80,), kappa=0.1)
    work = torch.zeros(256, dtype=torch.uint8, device="cuda")
    assert abi.otvmc_solve_snr(big.ans.handle, T, ns, z, z, z, z, z, 4.0, 1e-12, z, None, work, 256) == \
        abi.OTVMC_ERR_UNSUPPORTED
    c = Case((14,), kappa=0.1)  # P = 105: needs 2 P^2 doubles of workspace per trajectory
    assert abi.otvmc_solve_snr(c.ans.handle, T, ns, z, z, z, z, z, 4.0, 1e-12, z, None, work, 256) == \
        abi.OTVMC_ERR_WORKSPACE
    rbm = pkg.Ansatz(c.model, kind=abi.OTVMC_RBM, n_hidden=4)
    assert abi.otvmc_solve_snr(rbm.handle, T, ns, z, z, z, z, z, 4.0, 1e-12, z, None, work, 256) == \
        abi.OTVMC_ERR_UNSUPPORTED


@pytest.mark.parametrize("scheme,n", [(abi.OTVMC_HEUN, 8), (abi.OTVMC_MIDPOINT, 8), (abi.OTVMC_MIDPOINT, 16)])
def test_run_snr_matches_oracle(scheme, n):
    """Whole trajectories with the SNR regulariser (FP64): bit-identical chains and parameters
    that agree to 1e-9 with the oracle's MC otVMC driven by the same draws (P = 36 on the
    Jacobi path, P = 136 on the tridiagonal one)."""
    c = Case((n,), alpha=1.5, h=1.0, kappa=0.1)
    T, ns, steps, dt, seed = 2, 256, 3, 0.01, 91
    desc = abi.RunDesc(ntraj=T, traj0=0, ns=ns, n_steps=steps, step0=0, n_sweep=2, dt=dt, scheme=scheme,
                       precision=FP64, reg=abi.OTVMC_REG_SNR, eps=1e-4, snr_thresh=4.0, seed=seed,
                       measure_every=1, measure_final=1, use_graph=0)
    nmeas = abi.otvmc_run_n_meas(desc)
    theta = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    spins = torch.zeros((T, ns, c.W), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(c.ans.handle, T, 0, ns, seed, spins))
    nb = abi.otvmc_run_workspace_bytes(c.ans.handle, desc)
    assert nb > 0
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((nmeas, T, 9), dtype=torch.float64, device="cuda")
    check(abi.otvmc_run_trajectories(c.ans.handle, desc, theta, spins, mom, work, nb))
    sname = "heun" if scheme == abi.OTVMC_HEUN else "midpoint"
    oth, osig, om, oq = tr.run_mc(c.omodel, c.oans, T, ns, steps, dt, seed, sname, n_sweep=2, reg="snr")
    assert np.array_equal(unpack(spins, c.n), osig)
    assert rel_err(from_dev_complex(theta)[..., 0], oth) < 1e-9


def test_run_snr_rejects_large_P():
    c = Case((80,), kappa=0.1)  # P = 3240
    desc = abi.RunDesc(ntraj=1, traj0=0, ns=64, n_steps=1, step0=0, n_sweep=1, dt=0.01, scheme=abi.OTVMC_HEUN,
                       precision=FP64, reg=abi.OTVMC_REG_SNR, eps=1e-4, snr_thresh=4.0, seed=1,
                       measure_every=0, measure_final=0, use_graph=0)
    assert abi.otvmc_run_workspace_bytes(c.ans.handle, desc) == 0
