"""The partially inhomogeneous long-range Jastrow LJPHd / LJH (Eq. 12 and the paragraph after it)
on the GPU against the oracle's tied Jastrow: local estimators, S, obar and D of the tied
parameters, the regularised solves, whole trajectories with bit-identical Markov chains, and the
exact unitary Ising state that the homogeneous ansatz represents."""
import numpy as np
import pytest

from gpu_helpers import require_gpu, to_dev_complex, from_dev_complex, unpack, rel_err, torch
import synth
from oracle import tvmc, trajectories as tr
from oracle.ansatz import lj_ansatz
from oracle.model import Model as OModel, couplings
from paper_2506_23928_gb300 import abi
from paper_2506_23928_gb300.abi import check

pytestmark = pytest.mark.gpu
FP64, MIXED = abi.OTVMC_PREC_FP64, abi.OTVMC_PREC_MIXED


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


class LjCase:
    def __init__(self, n, d, pbc, alpha=1.5, h=0.9, kappa=0.1, gamma=0.05, J=1.0, kac=False):
        import paper_2506_23928_gb300 as pkg
        self.J = couplings((n,), J, alpha, kac=kac, pbc=pbc)
        self.n = n
        self.kappa = np.full(n, kappa)
        self.gamma = np.full(n, gamma)
        self.omodel = OModel(J=self.J, h=h, kappa=self.kappa, gamma=self.gamma)
        self.oans = lj_ansatz(n, d, pbc)
        self.model = pkg.Model(self.J, h, self.kappa, self.gamma)
        self.ans = pkg.Ansatz(self.model, kind=abi.OTVMC_LJ, d=d, pbc=pbc)
        self.P = self.ans.P
        self.nops = self.model.nops
        self.W = (n + 63) // 64
        assert self.P == self.oans.P

    def work(self, ntraj, ns, precision):
        nb = abi.otvmc_workspace_bytes(self.ans.handle, ntraj, ns, precision)
        assert nb > 0
        return torch.zeros(nb, dtype=torch.uint8, device="cuda"), nb


CASES = [(12, 1, False, 200), (11, 0, True, 64), (70, 2, False, 96), (20, 3, True, 136)]


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,d,pbc,ns", CASES)
def test_local_estimators(n, d, pbc, ns, precision):
    c = LjCase(n, d, pbc)
    T, dt = 2, 0.01
    th = synth.random_theta(11, T, c.P, 0.05)
    sig = synth.random_spins(12, T, ns, n)
    sp = torch.from_numpy(synth.pack_spins(sig).view(np.int64)).cuda()
    dW = synth.random_normals(13, (T, c.nops), np.sqrt(dt))
    E = torch.zeros((T, ns, 2), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(E)
    lpl = torch.zeros((T, c.nops), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, precision)
    check(abi.otvmc_local_estimators(c.ans.handle, to_dev_complex(th), sp, T, ns, torch.from_numpy(dW).cuda(), dt,
                                     precision, E, v, lpl, work, nb))
    check(abi.otvmc_check(work))
    E, v = from_dev_complex(E)[..., 0], from_dev_complex(v)[..., 0]
    tol = 1e-10 if precision == FP64 else 1e-5
    w = tvmc.mc_weights(ns)
    for t in range(T):
        terms = tvmc.local_terms(c.omodel, c.oans, th[t], sig[t])
        lp = tvmc.expectation(w, terms["LpLd"]).real
        Ew = tvmc.effective_energy(terms, lp)
        assert rel_err(E[t], Ew) < tol
        assert rel_err(v[t], -1j * dt * Ew + terms["B"] @ dW[t]) < tol
        assert rel_err(lpl.cpu().numpy()[t], lp) < tol


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,d,pbc,ns", CASES)
def test_build_S_D_and_solves(n, d, pbc, ns, precision):
    """S (FP64, from exact integer counts of the tied log-derivatives), obar and D (folded from
    the exact pair sums) against the oracle's covariances; the diagonal-shift solve and, for
    P <= 96, the SNR-filtered solve against the oracle's on the same S, D and samples."""
    c = LjCase(n, d, pbc)
    T, dt, eps = 2, 0.01, 1e-3
    th = synth.random_theta(21, T, c.P, 0.05)
    sig = synth.random_spins(22, T, ns, n)
    sp = torch.from_numpy(synth.pack_spins(sig).view(np.int64)).cuda()
    dW = synth.random_normals(23, (T, c.nops), np.sqrt(dt))
    w = tvmc.mc_weights(ns)
    evs = [tvmc.evaluate(c.omodel, c.oans, th[t], sig[t], w, dW[t], dt) for t in range(T)]
    v = np.stack([tvmc.local_v(evs[t], dW[t], dt) for t in range(T)])
    P = c.P
    S = torch.zeros((T, P, P), dtype=torch.float64, device="cuda")
    ob = torch.zeros((T, P), dtype=torch.float64, device="cuda")
    D = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, precision)
    check(abi.otvmc_build_S_F(c.ans.handle, None, sp, to_dev_complex(v), T, ns, precision, S, None, ob, D, work, nb))
    check(abi.otvmc_check(work))
    Sg, obg, Dg = S.cpu().numpy(), ob.cpu().numpy(), from_dev_complex(D)[..., 0]
    for t in range(T):
        assert rel_err(Sg[t], evs[t]["S"].real) < 1e-12
        assert np.abs(evs[t]["S"].imag).max() == 0.0
        assert rel_err(obg[t], evs[t]["O"].mean(axis=0).real) < 1e-13
        assert rel_err(Dg[t], evs[t]["D"]) < 1e-10
    delta = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    check(abi.otvmc_solve_step(c.ans.handle, T, ns, precision, abi.OTVMC_REG_SHIFT, eps, 4.0, S, None, ob, D, delta,
                               None, work, nb))
    check(abi.otvmc_check(work))
    got = from_dev_complex(delta)[..., 0]
    for t in range(T):
        assert rel_err(got[t], tvmc.solve_shift(evs[t]["S"], evs[t]["D"], eps)) < 1e-10
    if True:
        nbs = abi.otvmc_snr_workspace_bytes(c.ans.handle, T)
        works = torch.zeros(nbs, dtype=torch.uint8, device="cuda")
        check(abi.otvmc_solve_snr(c.ans.handle, T, ns, S, ob, sp, to_dev_complex(v), D, 4.0, 1e-12, delta, None,
                                  works, nbs))
        check(abi.otvmc_check(works))
        got = from_dev_complex(delta)[..., 0]
        for t in range(T):
            want = tvmc.solve_snr(evs[t]["S"], evs[t]["D"], evs[t]["O"], v[t], w, 4.0, 1e-12)
            assert rel_err(got[t], want) < 1e-8


def _run(c, T, ns, steps, dt, seed, precision, scheme, eps, reg=abi.OTVMC_REG_SHIFT, every=1, theta0=None):
    desc = abi.RunDesc(ntraj=T, traj0=0, ns=ns, n_steps=steps, step0=0, n_sweep=2, dt=dt, scheme=scheme,
                       precision=precision, reg=reg, eps=eps, snr_thresh=4.0, seed=seed, measure_every=every,
                       measure_final=1, use_graph=0)
    nm = abi.otvmc_run_n_meas(desc)
    th0 = np.zeros((T, c.P), complex) if theta0 is None else np.tile(theta0, (T, 1))
    theta = to_dev_complex(th0).reshape(T, c.P, 2)
    spins = torch.zeros((T, ns, c.W), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(c.ans.handle, T, 0, ns, seed, spins))
    nb = abi.otvmc_run_workspace_bytes(c.ans.handle, desc)
    assert nb > 0
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((nm, T, 9), dtype=torch.float64, device="cuda")
    check(abi.otvmc_run_trajectories(c.ans.handle, desc, theta, spins, mom, work, nb))
    check(abi.otvmc_check(work))
    return from_dev_complex(theta)[..., 0], unpack(spins, c.n), mom.cpu().numpy()


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,d,pbc,scheme,reg", [(10, 1, True, abi.OTVMC_HEUN, abi.OTVMC_REG_SHIFT),
                                                (10, 1, True, abi.OTVMC_MIDPOINT, abi.OTVMC_REG_SNR),
                                                (9, 0, False, abi.OTVMC_HEUN, abi.OTVMC_REG_SHIFT),
                                                (66, 1, True, abi.OTVMC_MIDPOINT, abi.OTVMC_REG_SHIFT),
                                                (66, 1, True, abi.OTVMC_HEUN, abi.OTVMC_REG_SNR)])
def test_run_matches_oracle(n, d, pbc, scheme, reg, precision):
    """Whole trajectories of the paper's setup (ring, alpha = 1 with the Kac factor, the LITF
    sign J_ij = -J/(K r), h -> -h, decay kappa = 0.5) from a random theta_0: identical chains,
    the parameter change within 1e-8 (FP64) or 1e-4 (mixed estimators) of its largest entry,
    moments within 1e-8 / 1e-5."""
    J, kappa = 1.0, 0.5
    c = LjCase(n, d, pbc, alpha=1.0, h=-0.3, kappa=kappa, gamma=0.0, J=-J, kac=True)
    T, ns, steps, dt, seed, eps = 2, 128 if n < 64 else 64, 3, 0.01, 808, 1e-3
    theta0 = synth.random_theta(9, 1, c.P, 0.05)[0]
    th, sig, mom = _run(c, T, ns, steps, dt, seed, precision, scheme, eps, reg, theta0=theta0)
    sname = "heun" if scheme == abi.OTVMC_HEUN else "midpoint"
    oth, osig, om, oq = tr.run_mc(c.omodel, c.oans, T, ns, steps, dt, seed, sname, n_sweep=2, eps=eps,
                                  theta0=theta0, reg="shift" if reg == abi.OTVMC_REG_SHIFT else "snr")
    assert np.array_equal(sig, osig)
    assert rel_err(th - theta0, oth - theta0) < (1e-8 if precision == FP64 else 1e-4)
    want = np.concatenate([om, oq[..., [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]], axis=-1)
    assert rel_err(mom, want) < (1e-8 if precision == FP64 else 1e-5)


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_homogeneous_ansatz_follows_the_exact_unitary_state(precision):
    """h = 0, no dissipation, ring of 32 spins: exp(-i t H) from +x is the LJH state
    eta_D = -i t J_D; after t = 1 (100 Heun steps) the 1 + 16 distance parameters stay within
    the sampling error of 4096 samples of it and <sigma^x> matches prod_k cos(2 J_jk t)."""
    n = 32
    c = LjCase(n, 0, True, alpha=1.5, h=0.0, kappa=0.0, gamma=0.0)
    assert c.P == n + n // 2
    steps, dt = 100, 0.01
    th, _, mom = _run(c, 4, 4096, steps, dt, 5, precision, abi.OTVMC_HEUN, 1e-4, every=0)
    Jd = np.array([c.J[0, D] for D in range(1, n // 2 + 1)])
    assert np.abs(th[:, n:] - (-1j * steps * dt * Jd)[None, :]).max() < 3e-4
    assert np.abs(th[:, :n]).max() < 1e-5
    mx_exact = np.prod(np.cos(2 * steps * dt * c.J[0, 1:]))
    assert np.abs(mom[-1, :, 0] - mx_exact).max() < 0.01


def test_full_limit_equals_the_jastrow_ansatz():
    """d = N - 1 gives the full Jastrow's parameters and results (to 1e-12) through the tied
    path (expanded parameters, integer Gram, FP64 solve) and the FP64 Jastrow path."""
    from gpu_helpers import Case
    n, T, ns, steps, dt, seed = 8, 2, 64, 2, 0.01, 3
    lj = LjCase(n, n - 1, False, alpha=1.5, h=1.0, kappa=0.1, gamma=0.0)
    full = Case((n,), alpha=1.5, h=1.0, kappa=0.1, gamma=0.0)
    assert lj.P == full.P
    th_l, sig_l, mom_l = _run(lj, T, ns, steps, dt, seed, FP64, abi.OTVMC_HEUN, 1e-4)
    th_f, sig_f, mom_f = _run(full, T, ns, steps, dt, seed, FP64, abi.OTVMC_HEUN, 1e-4)
    assert np.array_equal(sig_l, sig_f)
    assert rel_err(th_l, th_f) < 1e-12
    assert rel_err(mom_l, mom_f) < 1e-12
