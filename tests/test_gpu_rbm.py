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

    def work(self, ntraj, ns, precision=FP64, cap=None):
        nb = abi.otvmc_workspace_bytes(self.ans.handle, ntraj, ns, precision)
        assert nb > 0
        if cap is not None:
            nb = min(nb, cap)
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
@pytest.mark.parametrize("n,m,ns,gamma", [(7, 5, 300, 0.0), (10, 12, 96, 0.05), (64, 128, 40, 0.05),
                                         (256, 256, 32, 0.0)])  # the square16_rbm shape
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
    # the all-stage size holds the FP64 S of P = 66048 at the 16 x 16 shape; the estimators need
    # a small part of it (the call checks that what it carves fits)
    work, nb = c.work(T, ns, precision, cap=1 << 28)
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
    # the parameter change over the run, per element against its largest entry: 1e-8 on the
    # FP64 path, 1e-4 on the mixed path (the theta-dot tolerance of FP32-class paths)
    got = from_dev_complex(theta)[..., 0]
    tol = 1e-8 if precision == FP64 else 1e-4
    assert rel_err(got - theta0, oth - theta0) < tol
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


def _oracle_step(c, T, ns, dt, seed, eps, theta0):
    """One midpoint step of the oracle from theta0 on the same draws, the diagonal-shift solve
    taken through its Ns x Ns form (the same delta; S of P = 8384 or 66048 is not formed)."""
    oth, osig, _, _ = tr.run_mc(c.omodel, c.oans, T, ns, 1, dt, seed, "midpoint", n_sweep=2, eps=eps,
                                theta0=theta0, measure=False, push=True)
    return oth, osig


def _oracle_moments(c, theta, sig, chunk=8):
    """The oracle's per-trajectory moments, summed over chunks of samples (the two-flip ratios
    of an RBM take (chunk, N, N, M) entries); each chunk carries its weight 1/ns."""
    ns = sig.shape[0]
    w = np.full(ns, 1.0 / ns)
    m = np.zeros(3)
    q = np.zeros((3, 3))
    k = 0
    for x0 in range(0, ns, chunk):
        mm, qq = moments_from_samples(c.oans, theta, sig[x0:x0 + chunk], w[x0:x0 + chunk])
        m += mm
        q += qq
        k += 1
    q -= (k - 1) * np.eye(3) / c.n  # the same-site term 2 delta_ab is added once per call
    return np.concatenate([m, q[[0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]])


def _workload_theta0(c, seed, sd=0.01):
    """a = b = 0 and W ~ N(0, sd^2) in real and imaginary part, as the RBM workloads start."""
    g = synth.rng(seed)
    theta0 = np.zeros(c.P, complex)
    theta0[c.n + c.m:] = g.normal(0, sd, c.n * c.m) + 1j * g.normal(0, sd, c.n * c.m)
    return theta0


@pytest.mark.parametrize("tbuild", [FACT, MAT])
@pytest.mark.parametrize("ns", [256, 96])
def test_rbm_mixed_chain64_shape_matches_oracle(ns, tbuild):
    """The chain64_rbm shape (N = 64, M = 128, P = 8384 > ns: the T path, factored at size
    2 ns) with dephasing: one midpoint step of the mixed path (FP32 sampling and estimators, T
    from the factorised kernel or the split-BF16 tensor-core product of materialised O,
    tensor-core Cholesky, corrections against the exact operator) against the oracle on the
    same draws: identical chains, parameter change within 1e-4 of its largest entry, moments of
    the predictor samples within 1e-5.  Shift 1e-4 (the workloads') for the factorised T; 1e-3
    for the materialised product, whose FP32 sums over K = 2P products leave an error of
    ~1e-5 |T| that the corrections remove only while it is well below the shift."""
    c = RbmCase(64, 128, gamma=0.05)
    check(abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, tbuild))
    T, dt, seed, eps = 2, 0.005, 99, (1e-4 if tbuild == FACT else 1e-3)
    theta0 = synth.random_theta(5, 1, c.P, 0.01)[0]
    th_m, sp_m, mo_m = _run(c, MIXED, T, ns, 1, dt, seed, eps, theta0)
    oth, osig = _oracle_step(c, T, ns, dt, seed, eps, theta0)
    e = rel_err(th_m - theta0, oth - theta0)
    assert np.array_equal(sp_m, osig), e
    assert e < 1e-4, e
    if ns <= 96:
        from oracle.philox import initial_spins
        for t in range(T):
            sig0, _ = tvmc.metropolis(c.oans, theta0, initial_spins(seed, t, ns, c.n), seed, t, 0, 2)
            assert rel_err(mo_m[0, t], _oracle_moments(c, theta0, sig0)) < 1e-5


@pytest.mark.parametrize("n,m,ns", [(64, 128, 200), (70, 20, 136), (5, 9, 40)])
def test_rbm_factored_and_materialised_t_match_oracle(n, m, ns):
    """One step's parameter change on the T path from the factorised T (no O in memory) and
    from the split-BF16 product of materialised O, both against the oracle on the same draws
    (two words of spins for N = 70, ragged sample tiles for ns = 136, 200, 40), within 1e-4;
    shift 1e-4 for the factorised T, 1e-3 for the materialised product (its FP32 sums over
    K = 2P products)."""
    c = RbmCase(n, m, gamma=0.05)
    assert c.P > ns
    T, dt, seed = 3, 0.005, 31
    theta0 = synth.random_theta(8, 1, c.P, 0.05)[0]
    for tb, eps in ((FACT, 1e-4), (MAT, 1e-3)):
        oth, osig = _oracle_step(c, T, ns, dt, seed, eps, theta0)
        check(abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, tb))
        th, sp, _ = _run(c, MIXED, T, ns, 1, dt, seed, eps, theta0)
        e = rel_err(th - theta0, oth - theta0)
        assert np.array_equal(sp, osig), (tb, e)
        assert e < 1e-4, (tb, e)


def test_rbm_t_build_option_validation():
    c = RbmCase(4, 3)
    assert abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, 2) == abi.OTVMC_ERR_INVALID
    assert abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, MAT) == abi.OTVMC_OK
    from gpu_helpers import Case
    j = Case((4,))
    assert abi.otvmc_ansatz_set_rbm_t_build(j.ans.handle, FACT) == abi.OTVMC_ERR_INVALID


@pytest.mark.parametrize("workload,ns,T", [("chain64_rbm", 2048, 1), ("square16_rbm", 128, 2)])
def test_rbm_mixed_workload_shape_matches_oracle(workload, ns, T):
    """The RBM workloads' models and ansatz shapes with the workloads' shift 1e-4 and initial
    weights N(0, 0.01^2): chain64_rbm (N = 64, M = 128, P = 8384) at ns = 2048, the smallest
    sample count of its mix (T path of size 4096), and square16_rbm (16 x 16 lattice, N = M = 256,
    P = 66048) at ns = 128.  One midpoint step of the mixed path (factorised T) against the
    oracle on the same draws: identical chains, parameter change within 1e-4."""
    w = synth.WORKLOADS[workload]
    import paper_2506_23928_gb300 as pkg
    c = RbmCase.__new__(RbmCase)
    c.J = couplings(w.extent, w.J, w.alpha)
    c.n, c.m = w.n, w.n_hidden
    c.kappa, c.gamma = np.full(c.n, w.kappa), np.full(c.n, w.gamma)
    c.omodel = OModel(J=c.J, h=w.h, kappa=c.kappa, gamma=c.gamma)
    c.oans = RBM(c.n, c.m)
    c.model = pkg.Model(c.J, w.h, c.kappa, c.gamma)
    c.ans = pkg.Ansatz(c.model, kind=abi.OTVMC_RBM, n_hidden=c.m)
    c.P, c.nops, c.W = c.ans.P, c.model.nops, (c.n + 63) // 64
    check(abi.otvmc_ansatz_set_rbm_t_build(c.ans.handle, FACT))
    seed = 7
    theta0 = _workload_theta0(c, 11)
    th_m, sp_m, _ = _run(c, MIXED, T, ns, 1, w.dt, seed, w.eps, theta0)
    oth, osig = _oracle_step(c, T, ns, w.dt, seed, w.eps, theta0)
    e = rel_err(th_m - theta0, oth - theta0)
    assert np.array_equal(sp_m, osig), e
    assert e < 1e-4, e
