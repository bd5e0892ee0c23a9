"""RBM ansatz (Eq. 11) on the FP64 path, stage by stage and whole trajectories, against the
oracle's RBM (complex log-derivatives, complex Hermitian S) on the same inputs; both the S
path (P <= ns) and the push-through T path (P > ns) of the solve."""
import numpy as np
import pytest

from gpu_helpers import require_gpu, to_dev_complex, from_dev_complex, unpack, rel_err, torch
import synth
from oracle import tvmc, trajectories as tr
from oracle.ansatz import RBM
from oracle.model import Model as OModel, couplings
from oracle.observables import moments_from_samples
from paper_2506_23928_gb300 import abi
from paper_2506_23928_gb300.abi import check

pytestmark = pytest.mark.gpu
FP64, MIXED = abi.OTVMC_PREC_FP64, abi.OTVMC_PREC_MIXED
FACT, MAT = abi.OTVMC_RBM_T_FACTORED, abi.OTVMC_RBM_T_MATERIALISED
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


class RbmCase:
    def __init__(self, n, m, h=0.9, kappa=0.1, gamma=0.0, alpha=1.5):
        import paper_2506_23928_gb300 as pkg
        self.J = couplings((n,), 1.0, alpha)
        self.n, self.m = n, m
        self.kappa = np.full(n, kappa)
        self.gamma = np.full(n, gamma)
        self.omodel = OModel(J=self.J, h=h, kappa=self.kappa, gamma=self.gamma)
        self.oans = RBM(n, m)
        self.model = pkg.Model(self.J, h, self.kappa, self.gamma)
        self.ans = pkg.Ansatz(self.model, kind=abi.OTVMC_RBM, n_hidden=m)
        self.P = self.ans.P
        self.nops = self.model.nops
        self.W = (n + 63) // 64
        assert self.P == self.oans.P == n + m + n * m

    def theta(self, seed, ntraj, scale):
        th = synth.random_theta(seed, ntraj, self.P, scale)
        return th, to_dev_complex(th)

    def spins(self, seed, ntraj, ns):
        sig = synth.random_spins(seed, ntraj, ns, self.n)
        return sig, torch.from_numpy(synth.pack_spins(sig).view(np.int64)).cuda()

    def work(self, ntraj, ns, precision=FP64):
        nb = abi.otvmc_workspace_bytes(self.ans.handle, ntraj, ns, precision)
        assert nb > 0
        return torch.zeros(nb, dtype=torch.uint8, device="cuda"), nb


@pytest.mark.parametrize("n,m,ns,scale", [(6, 4, 150, 0.3), (9, 7, 64, 0.3), (70, 3, 40, 0.3),
                                          (64, 128, 48, 0.05),   # the chain64_rbm shape (FP32 warp sampler)
                                          (12, 40, 200, 1.0),    # large parameters: many decisions near the band
                                          (9, 200, 40, 0.1),     # 8 hidden units per lane, W in shared memory
                                          (200, 100, 24, 0.05),  # 4 per lane, W (160 KB) read from theta
                                          (256, 256, 16, 0.02),  # the square16_rbm shape
                                          (4, 300, 64, 0.2)])    # M > 256: the FP64 sampler
def test_rbm_sample_bit_exact(n, m, ns, scale):
    """Every accept/reject equals the FP64 decision (FP32 sampler with its error bound and
    FP64 recompute inside the band; FP64 sampler beyond 256 hidden units)."""
    c = RbmCase(n, m)
    T, traj0, seed, ev, sweeps = 2, 3, 77, 5, 2
    th, th_d = c.theta(1, T, scale)
    sig, sp = c.spins(2, T, ns)
    acc = torch.zeros(T, dtype=torch.int64, device="cuda")
    # the sampler's own scratch (the FP64 sampler's angles and Re lc, the FP32 sampler's tables
    # of flip factors, W and a), not the all-stage size, which for the 16 x 16 shape holds the
    # FP64 S of P = 66048
    nb = T * m * ns * 24 + T * n * (40 * m + 8) + 65536
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    check(abi.otvmc_sample(c.ans.handle, th_d, T, traj0, ns, sweeps, seed, ev, sp, acc, work, nb))
    check(abi.otvmc_check(work))
    got = unpack(sp, n)
    for t in range(T):
        want, a = tvmc.metropolis(c.oans, th[t], sig[t], seed, traj0 + t, ev, sweeps)
        assert np.array_equal(got[t], want)
        assert int(acc[t]) == int(a.sum())


def _evaluate(c, T, ns, seed, scale, dt):
    th, th_d = c.theta(seed, T, scale)
    sig, sp = c.spins(seed + 1, T, ns)
    dW = synth.random_normals(seed + 2, (T, c.nops), np.sqrt(dt))
    w = tvmc.mc_weights(ns)
    evs = [tvmc.evaluate(c.omodel, c.oans, th[t], sig[t], w, dW[t], dt) for t in range(T)]
    return th, th_d, sig, sp, dW, evs


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,m,ns,gamma", [(7, 5, 300, 0.0), (10, 12, 96, 0.05), (64, 128, 40, 0.05)])
def test_rbm_local_estimators(precision, n, m, ns, gamma):
    """E_eff, v and <L+L^+> against the oracle's local terms (FP64 1e-10, mixed 1e-5)."""
    c = RbmCase(n, m, gamma=gamma)
    T, dt = 2, 0.01
    th, th_d = c.theta(11, T, 0.2 if n < 64 else 0.03)
    sig, sp = c.spins(12, T, ns)
    dW = synth.random_normals(13, (T, c.nops), np.sqrt(dt))
    dW_d = torch.from_numpy(dW).cuda()
    E = torch.zeros((T, ns, 2), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(E)
    lpl = torch.zeros((T, max(c.nops, 1)), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, precision)
    check(abi.otvmc_local_estimators(c.ans.handle, th_d, sp, T, ns, dW_d, dt, precision, E, v, lpl, work, nb))
    check(abi.otvmc_check(work))
    E, v = from_dev_complex(E)[..., 0], from_dev_complex(v)[..., 0]
    tol = TOL if precision == FP64 else 1e-5
    w = tvmc.mc_weights(ns)
    for t in range(T):
        terms = tvmc.local_terms(c.omodel, c.oans, th[t], sig[t])
        lp = tvmc.expectation(w, terms["LpLd"]).real
        Ew = tvmc.effective_energy(terms, lp)
        assert rel_err(E[t], Ew) < tol
        assert rel_err(v[t], -1j * dt * Ew + terms["B"] @ dW[t]) < tol
        assert rel_err(lpl.cpu().numpy()[t, :c.nops], lp) < tol


@pytest.mark.parametrize("n,m,ns", [(6, 4, 200), (5, 9, 40)])
def test_rbm_build_and_solve(n, m, ns):
    """Complex Hermitian S, complex obar and D, then (S + eps I) delta = D through the real
    embedding, including P > ns (S singular, only the shift makes it definite)."""
    c = RbmCase(n, m, gamma=0.05)
    T, dt, eps = 2, 0.01, 1e-3
    th, th_d, sig, sp, dW, evs = _evaluate(c, T, ns, 21, 0.2, dt)
    v = np.stack([tvmc.local_v(evs[t], dW[t], dt) for t in range(T)])
    P = c.P
    S = torch.zeros((T, P, P, 2), dtype=torch.float64, device="cuda")
    ob = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    D = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns)
    check(abi.otvmc_build_S_F(c.ans.handle, th_d, sp, to_dev_complex(v), T, ns, FP64, S, None, ob, D, work, nb))
    check(abi.otvmc_check(work))
    Sg, obg, Dg = from_dev_complex(S)[..., 0], from_dev_complex(ob)[..., 0], from_dev_complex(D)[..., 0]
    for t in range(T):
        assert rel_err(Sg[t], evs[t]["S"]) < 1e-12
        assert rel_err(obg[t], evs[t]["O"].mean(axis=0)) < 1e-13
        assert rel_err(Dg[t], evs[t]["D"]) < 1e-11
    delta = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    shift = torch.zeros(T, dtype=torch.float64, device="cuda")
    check(abi.otvmc_solve_step(c.ans.handle, T, ns, FP64, abi.OTVMC_REG_SHIFT, eps, 4.0, S, None, None, D, delta,
                               shift, work, nb))
    check(abi.otvmc_check(work))
    got = from_dev_complex(delta)[..., 0]
    for t in range(T):
        assert rel_err(got[t], tvmc.solve_shift(evs[t]["S"], evs[t]["D"], eps)) < 1e-9
        assert float(shift[t]) == eps


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,m,ns", [(6, 3, 100), (4, 5, 33)])
def test_rbm_observables(precision, n, m, ns):
    c = RbmCase(n, m)
    T = 2
    th, th_d = c.theta(31, T, 0.3)
    sig, sp = c.spins(32, T, ns)
    mom = torch.zeros((T, 9), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, precision)
    check(abi.otvmc_observables(c.ans.handle, th_d, sp, T, ns, precision, mom, work, nb))
    check(abi.otvmc_check(work))
    got = mom.cpu().numpy()
    for t in range(T):
        mm, q = moments_from_samples(c.oans, th[t], sig[t], tvmc.mc_weights(ns))
        want = np.concatenate([mm, q[[0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]])
        assert rel_err(got[t], want) < (TOL if precision == FP64 else 1e-5)


@pytest.mark.parametrize("n,m,ns,scheme", [(6, 4, 128, abi.OTVMC_HEUN),     # S path, P = 34 <= ns
                                          (6, 4, 24, abi.OTVMC_MIDPOINT),   # T path, P = 34 > ns
                                          (5, 6, 16, abi.OTVMC_HEUN)])      # T path, P = 41
@pytest.mark.parametrize("precision,tbuild", [(FP64, FACT), (MIXED, FACT), (MIXED, MAT)])
def test_rbm_run_matches_oracle(n, m, ns, scheme, precision, tbuild):
    """Whole trajectories with decay and dephasing from a random theta_0 (from theta = 0 the
    hidden biases and weights of an RBM stay zero: tanh 0 = 0 makes their log-derivatives
    vanish), bit-identical chains and parameters within 1e-8 of the oracle, whose solve
    always goes through S; on the T path the push-through identity gives the same delta,
    with T formed from the factorised kernel or from materialised O on the mixed path."""
    c = RbmCase(n, m, gamma=0.05)
    check(abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, tbuild))
    T, steps, dt, seed, eps = 2, 3, 0.01, 4242, 1e-3
    theta0 = synth.random_theta(77, 1, c.P, 0.1)[0]
    desc = abi.RunDesc(ntraj=T, traj0=0, ns=ns, n_steps=steps, step0=0, n_sweep=2, dt=dt, scheme=scheme,
                       precision=precision, reg=abi.OTVMC_REG_SHIFT, eps=eps, snr_thresh=4.0, seed=seed,
                       measure_every=1, measure_final=1, use_graph=0)
    nmeas = abi.otvmc_run_n_meas(desc)
    theta = to_dev_complex(np.tile(theta0, (T, 1))).reshape(T, c.P, 2)
    spins = torch.zeros((T, ns, c.W), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(c.ans.handle, T, 0, ns, seed, spins))
    nb = abi.otvmc_run_workspace_bytes(c.ans.handle, desc)
    assert nb > 0
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((nmeas, T, 9), dtype=torch.float64, device="cuda")
    check(abi.otvmc_run_trajectories(c.ans.handle, desc, theta, spins, mom, work, nb))
    sname = "heun" if scheme == abi.OTVMC_HEUN else "midpoint"
    oth, osig, om, oq = tr.run_mc(c.omodel, c.oans, T, ns, steps, dt, seed, sname, n_sweep=2, eps=eps,
                                  theta0=theta0)
    assert np.abs(oth[:, c.n + c.m:] - theta0[c.n + c.m:]).max() > 1e-6  # the weights moved
    assert np.array_equal(unpack(spins, c.n), osig)
    # the mixed path's S or T is an FP32 sum of split-BF16 products (not exact as for the
    # Jastrow +-1 counts), so its solve carries ~kappa x 1e-7 relative error: 3e-4 of max|theta|
    tol = 1e-8 if precision == FP64 else 3e-4
    assert rel_err(from_dev_complex(theta)[..., 0], oth) < tol
    want = np.concatenate([om, oq[..., [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]], axis=-1)
    assert rel_err(mom.cpu().numpy(), want) < (1e-8 if precision == FP64 else 1e-4)


def test_rbm_mixed_run_rejected_beyond_256_hidden():
    c = RbmCase(4, 300)
    desc = abi.RunDesc(ntraj=1, traj0=0, ns=64, n_steps=1, step0=0, n_sweep=1, dt=0.01, scheme=abi.OTVMC_HEUN,
                       precision=MIXED, reg=abi.OTVMC_REG_SHIFT, eps=1e-4, snr_thresh=4.0, seed=1,
                       measure_every=0, measure_final=0, use_graph=0)
    assert abi.otvmc_run_workspace_bytes(c.ans.handle, desc) == 0
    desc.precision = FP64
    assert abi.otvmc_run_workspace_bytes(c.ans.handle, desc) > 0


def _run(c, precision, T, ns, steps, dt, seed, eps, theta0):
    desc = abi.RunDesc(ntraj=T, traj0=0, ns=ns, n_steps=steps, step0=0, n_sweep=2, dt=dt, scheme=abi.OTVMC_MIDPOINT,
                       precision=precision, reg=abi.OTVMC_REG_SHIFT, eps=eps, snr_thresh=4.0, seed=seed,
                       measure_every=1, measure_final=0, use_graph=0)
    theta = to_dev_complex(np.tile(theta0, (T, 1))).reshape(T, c.P, 2)
    spins = torch.zeros((T, ns, c.W), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(c.ans.handle, T, 0, ns, seed, spins))
    nb = abi.otvmc_run_workspace_bytes(c.ans.handle, desc)
    assert nb > 0
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((abi.otvmc_run_n_meas(desc), T, 9), dtype=torch.float64, device="cuda")
    check(abi.otvmc_run_trajectories(c.ans.handle, desc, theta, spins, mom, work, nb))
    return from_dev_complex(theta)[..., 0], unpack(spins, c.n), mom.cpu().numpy()


@pytest.mark.parametrize("tbuild", [FACT, MAT])
@pytest.mark.parametrize("ns", [256, 96])
def test_rbm_mixed_tensor_core_path_chain64_shape(ns, tbuild):
    """The chain64_rbm shape (N = 64, M = 128, P = 8384 > ns: the T path, factored at size
    2 ns): the mixed path (FP32 sampling and estimators, T from the factorised kernel or the
    split-BF16 tensor-core product of materialised O, tensor-core Cholesky with refinement)
    against the FP64 path on the same draws."""
    c = RbmCase(64, 128, gamma=0.05)
    check(abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, tbuild))
    T, steps, dt, seed, eps = 2, 1, 0.005, 99, 1e-3
    theta0 = synth.random_theta(5, 1, c.P, 0.01)[0]
    th_m, sp_m, mo_m = _run(c, MIXED, T, ns, steps, dt, seed, eps, theta0)
    th_f, sp_f, mo_f = _run(c, FP64, T, ns, steps, dt, seed, eps, theta0)
    # the parameter change of one step (measured ~2e-4 relative: FP32-accumulated T, eps 1e-3)
    assert rel_err(th_m - theta0, th_f - theta0) < 1e-3
    assert rel_err(mo_m, mo_f) < 1e-5  # moments of the predictor samples (identical chains at theta_0)


def test_rbm_t_build_option_validation():
    c = RbmCase(4, 3)
    assert abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, 2) == abi.OTVMC_ERR_INVALID
    assert abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, MAT) == abi.OTVMC_OK
    from gpu_helpers import Case
    j = Case((4,))
    assert abi.otvmc_ansatz_set_rbm_t_build(j.ans.handle, FACT) == abi.OTVMC_ERR_INVALID


@pytest.mark.parametrize("n,m,ns", [(64, 128, 200), (70, 20, 136), (5, 9, 40)])
def test_rbm_factored_t_equals_materialised(n, m, ns):
    """One evaluation's parameter change on the T path from the factorised T (no O in memory)
    and from the split-BF16 product of materialised O, both against the FP64 path on the same
    draws (two words of spins for N = 70, ragged sample tiles for ns = 136, 200, 40)."""
    c = RbmCase(n, m, gamma=0.05)
    assert c.P > ns
    T, dt, seed, eps = 3, 0.005, 31, 1e-3
    theta0 = synth.random_theta(8, 1, c.P, 0.05)[0]
    res = {}
    for tb in (FACT, MAT):
        check(abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, tb))
        res[tb] = _run(c, MIXED, T, ns, 1, dt, seed, eps, theta0)
    th_d, sp_d, _ = _run(c, FP64, T, ns, 1, dt, seed, eps, theta0)
    th_f, sp_f, _ = res[FACT]
    th_m, sp_m, _ = res[MAT]
    assert np.array_equal(sp_f, sp_d) and np.array_equal(sp_m, sp_d)
    assert rel_err(th_f - theta0, th_d - theta0) < 1e-3
    assert rel_err(th_m - theta0, th_d - theta0) < 1e-3


def test_rbm_mixed_full_size_chain64_rbm():
    """The chain64_rbm configuration the benchmark times (N = 64, M = 128, P = 8384, N_s = 2048,
    T path of size 4096, weights N(0, 0.01^2), shift 1e-4 as in the workload): one trajectory step of
    the mixed path (factorised T) against the FP64 path on the same draws, on two trajectories:
    identical chains, parameter change within 1e-3, moments within 1e-5."""
    w = synth.WORKLOADS["chain64_rbm"]
    c = RbmCase(w.n, w.n_hidden, h=w.h, kappa=w.kappa, gamma=w.gamma, alpha=w.alpha)
    check(abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, FACT))
    T, ns, seed = 2, 2048, 7
    g = synth.rng(11)
    theta0 = np.zeros(c.P, complex)
    theta0[c.n + c.m:] = g.normal(0, 0.01, c.n * c.m) + 1j * g.normal(0, 0.01, c.n * c.m)
    th_m, sp_m, mo_m = _run(c, MIXED, T, ns, 1, w.dt, seed, w.eps, theta0)
    th_f, sp_f, mo_f = _run(c, FP64, T, ns, 1, w.dt, seed, w.eps, theta0)
    assert np.array_equal(sp_m, sp_f)
    e = rel_err(th_m - theta0, th_f - theta0)
    assert e < 1e-3, e
    assert rel_err(mo_m, mo_f) < 1e-5
