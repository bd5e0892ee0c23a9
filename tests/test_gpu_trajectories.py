"""Whole trajectories through otvmc_run_trajectories against the oracle's MC otVMC driven
by the same counter-based draws, plus sampled checks at the benchmark's full size."""
import numpy as np
import pytest

from gpu_helpers import Case, require_gpu, to_dev_complex, from_dev_complex, unpack, rel_err, torch
import synth
from oracle import philox, tvmc, trajectories as tr
from paper_2506_23928_gb300 import abi
from paper_2506_23928_gb300.abi import check

pytestmark = pytest.mark.gpu
FP64, MIXED = abi.OTVMC_PREC_FP64, abi.OTVMC_PREC_MIXED


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def run_gpu(c, T, ns, steps, dt, seed, scheme, precision, eps=1e-4, sweeps=2, traj0=0, host=False):
    desc = abi.RunDesc(ntraj=T, traj0=traj0, ns=ns, n_steps=steps, step0=0, n_sweep=sweeps, dt=dt, scheme=scheme,
                       precision=precision, reg=abi.OTVMC_REG_SHIFT, eps=eps, snr_thresh=4.0, seed=seed,
                       measure_every=1, measure_final=1, use_graph=0)
    nmeas = abi.otvmc_run_n_meas(desc)
    theta = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    spins = torch.zeros((T, ns, c.W), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(c.ans.handle, T, traj0, ns, seed, spins))
    if host:
        nb = abi.otvmc_run_host_workspace_bytes(c.ans.handle, desc)
        work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        th_h = theta.cpu().contiguous()
        sp_h = spins.cpu().contiguous()
        mo_h = torch.zeros((nmeas, T, 9), dtype=torch.float64)
        check(abi.otvmc_run_trajectories_host(c.ans.handle, desc, th_h, sp_h, mo_h, work, nb))
        return from_dev_complex(th_h)[..., 0], unpack(sp_h, c.n), mo_h.numpy()
    nb = abi.otvmc_run_workspace_bytes(c.ans.handle, desc)
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((nmeas, T, 9), dtype=torch.float64, device="cuda")
    check(abi.otvmc_run_trajectories(c.ans.handle, desc, theta, spins, mom, work, nb))
    return from_dev_complex(theta)[..., 0], unpack(spins, c.n), mom.cpu().numpy()


def oracle_moments(m, q):
    return np.concatenate([m, q[..., [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]], axis=-1)


@pytest.mark.parametrize("precision,scheme", [(FP64, abi.OTVMC_HEUN), (MIXED, abi.OTVMC_HEUN),
                                              (FP64, abi.OTVMC_MIDPOINT), (MIXED, abi.OTVMC_MIDPOINT)])
def test_run_matches_oracle_chain8(precision, scheme):
    """Chain of 8 spins (the small benchmark workload's model), a few steps."""
    c = Case((8,), alpha=1.5, h=1.0, kappa=0.1)
    T, ns, steps, dt, seed = 3, 256, 3, 0.01, 77
    th, sp, mom = run_gpu(c, T, ns, steps, dt, seed, scheme, precision)
    sname = "heun" if scheme == abi.OTVMC_HEUN else "midpoint"
    oth, osig, om, oq = tr.run_mc(c.omodel, c.oans, T, ns, steps, dt, seed, sname, n_sweep=2, eps=1e-4)
    assert np.array_equal(sp, osig)
    tol = 1e-9 if precision == FP64 else 1e-4
    assert rel_err(th, oth) < tol
    assert rel_err(mom, oracle_moments(om, oq)) < (1e-9 if precision == FP64 else 1e-5)


def test_run_matches_oracle_dephasing_and_two_words():
    """65 spins (two spin words), decay and dephasing, midpoint, FP64 path.

    Bit-identical chains need parameters that agree to ~1e-12: with ns = 64 < P the shifted
    S has a condition number near 1e5, so this comparison runs on the FP64 path."""
    c = Case((65,), alpha=1.5, h=1.0, kappa=0.1, gamma=0.05)
    T, ns, steps, dt, seed = 2, 64, 2, 0.005, 5
    th, sp, mom = run_gpu(c, T, ns, steps, dt, seed, abi.OTVMC_MIDPOINT, FP64, traj0=3)
    oth, osig, om, oq = tr.run_mc(c.omodel, c.oans, T, ns, steps, dt, seed, "midpoint", n_sweep=2, eps=1e-4,
                                  traj0=3)
    assert np.array_equal(sp, osig)
    assert rel_err(th, oth) < 1e-8
    assert rel_err(mom, oracle_moments(om, oq)) < 1e-9


def test_run_host_buffers_equal_device_run():
    c = Case((8,), kappa=0.1)
    a = run_gpu(c, 2, 64, 2, 0.01, 9, abi.OTVMC_HEUN, MIXED)
    b = run_gpu(c, 2, 64, 2, 0.01, 9, abi.OTVMC_HEUN, MIXED, host=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_batching_does_not_change_results():
    """Counter-based draws keyed by the global trajectory id: a batch of 4 equals 2 + 2."""
    c = Case((10,), kappa=0.1)
    full = run_gpu(c, 4, 64, 2, 0.01, 3, abi.OTVMC_HEUN, MIXED)
    lo = run_gpu(c, 2, 64, 2, 0.01, 3, abi.OTVMC_HEUN, MIXED, traj0=0)
    hi = run_gpu(c, 2, 64, 2, 0.01, 3, abi.OTVMC_HEUN, MIXED, traj0=2)
    assert np.array_equal(full[0], np.concatenate([lo[0], hi[0]]))
    assert np.array_equal(full[1], np.concatenate([lo[1], hi[1]]))


def test_pipelined_batch_equals_separate_batches():
    """A batch of 40 trajectories runs as two sub-batches of 20 on forked streams (the solver's
    trajectory groups forked again inside each); it equals a batch of 24 and a batch of 16 run
    apart, in theta, spins and every measured moment, with device and host buffers, and with the
    sub-batches serialised on the caller's stream (serial profiling)."""
    c = Case((10,), kappa=0.1)
    args = (64, 2, 0.01, 3, abi.OTVMC_HEUN, MIXED)
    full = run_gpu(c, 40, *args)
    lo = run_gpu(c, 24, *args, traj0=0)
    hi = run_gpu(c, 16, *args, traj0=24)
    assert np.array_equal(full[0], np.concatenate([lo[0], hi[0]]))
    assert np.array_equal(full[1], np.concatenate([lo[1], hi[1]]))
    assert np.array_equal(full[2], np.concatenate([lo[2], hi[2]], axis=1))
    host = run_gpu(c, 40, *args, host=True)
    abi.otvmc_profile_enable(abi.OTVMC_PROFILE_SERIAL)
    try:
        ser = run_gpu(c, 40, *args)
        prof = abi.profile_summary()
    finally:
        abi.otvmc_profile_enable(abi.OTVMC_PROFILE_OFF)
    for k in range(3):
        assert np.array_equal(full[k], host[k])
        assert np.array_equal(full[k], ser[k])
    assert prof["sample"][1] > 0


def test_full_size_run_is_batch_invariant():
    """The benchmark's launch configuration: 256 trajectories of the 64-spin workload (P = 2080,
    N_s = 4096) through otvmc_run_trajectories, i.e. two sub-batches of 128 whose solves run as
    groups of 64.  The same trajectories run as a batch of 128 (two sub-batches of 64, four
    solver groups of 16 each) and as a batch of 16 (one batch, four groups of 4) give the same
    theta, chains and moments bit for bit."""
    c = Case((64,), alpha=1.5, h=1.0, kappa=0.1, gamma=0.05)
    args = (4096, 1, 0.005, 2026, abi.OTVMC_MIDPOINT, MIXED)
    full = run_gpu(c, 256, *args)
    for T, t0 in ((128, 0), (16, 240)):
        part = run_gpu(c, T, *args, traj0=t0)
        assert np.array_equal(full[0][t0:t0 + T], part[0])
        assert np.array_equal(full[1][t0:t0 + T], part[1])
        assert np.array_equal(full[2][:, t0:t0 + T], part[2])
    assert np.all(np.isfinite(full[0])) and np.abs(full[0]).max() > 0


def test_full_size_chain64_sampled():
    """The benchmark launch shape (N = 64, P = 2080, ns = 4096, 256 trajectories): one
    evaluation's sampler, S, D and solve, checked on sampled trajectories and entries."""
    c = Case((64,), alpha=1.5, h=1.0, kappa=0.1, gamma=0.05)
    T, ns, dt, eps, seed = 256, 4096, 0.005, 1e-4, 2026
    th, th_d = c.theta(71, T, 0.03)
    sig0, sp = c.spins(72, T, ns)
    work, nb = c.work(T, ns, MIXED)
    check(abi.otvmc_sample(c.ans.handle, th_d, T, 0, ns, 2, seed, 0, sp, None, work, nb))
    sig = unpack(sp, c.n)
    # sampler: 48 chains of two trajectories, bit for bit
    for t in (5, 200):
        ids = np.arange(0, ns, ns // 48)[:48]
        want, _ = tvmc.metropolis(c.oans, th[t], sig0[t][ids], seed, t, 0, 2, chain_ids=ids)
        assert np.array_equal(sig[t][ids], want)
    dW = synth.random_normals(73, (T, c.nops), np.sqrt(dt))
    dW_d = torch.from_numpy(dW).cuda()
    E = torch.zeros((T, ns, 2), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(E)
    check(abi.otvmc_local_estimators(c.ans.handle, th_d, sp, T, ns, dW_d, dt, MIXED, E, v, None, work, nb))
    G = torch.zeros((T, c.P, c.P), dtype=torch.float32, device="cuda")
    ob = torch.zeros((T, c.P), dtype=torch.float64, device="cuda")
    D = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    check(abi.otvmc_build_S_F(c.ans.handle, None, sp, v, T, ns, MIXED, None, G, ob, D, work, nb))
    delta = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    del work
    work, nb = c.work(T, ns, MIXED)
    check(abi.otvmc_solve_step(c.ans.handle, T, ns, MIXED, abi.OTVMC_REG_SHIFT, eps, 4.0, None, G, ob, D, delta,
                               None, work, nb))
    check(abi.otvmc_check(work))
    vv = from_dev_complex(v)[..., 0]
    Dg = from_dev_complex(D)[..., 0]
    dg = from_dev_complex(delta)[..., 0]
    for t in (5, 200):
        s = sig[t]
        ev = tvmc.evaluate(c.omodel, c.oans, th[t], s, tvmc.mc_weights(ns), dW[t], dt)
        assert rel_err(vv[t], tvmc.local_v(ev, dW[t], dt)) < 1e-5
        Gt = G[t].cpu().numpy()
        S_gpu = np.triu(Gt) / ns
        S_gpu = S_gpu + np.triu(S_gpu, 1).T - np.outer(ob[t].cpu().numpy(), ob[t].cpu().numpy())
        assert rel_err(S_gpu, ev["S"].real) < 1e-12
        assert rel_err(Dg[t], ev["D"]) < 1e-5
        assert rel_err(dg[t], tvmc.solve_shift(ev["S"], ev["D"], eps)) < 1e-4


def test_full_size_square10_sampled():
    """The 10 x 10 lattice workload at full size (N = 100, P = 5050, ns = 8192: 40 block
    columns, the last 58 wide; two spin words): sampled chains bit for bit, E_eff and v on
    sampled trajectories, sampled entries of G, obar and D from their definitions, and the
    mixed solve against an FP64 Cholesky solve of the same system."""
    import scipy.linalg
    c = Case((10, 10), alpha=3.0, h=0.5, kappa=0.05)
    T, ns, dt, eps, seed = 4, 8192, 0.005, 1e-4, 2027
    assert c.P == 5050 and c.W == 2
    th, th_d = c.theta(81, T, 0.02)
    sig0, sp = c.spins(82, T, ns)
    work, nb = c.work(T, ns, MIXED)
    check(abi.otvmc_sample(c.ans.handle, th_d, T, 0, ns, 2, seed, 0, sp, None, work, nb))
    sig = unpack(sp, c.n)
    ids = np.arange(0, ns, ns // 32)[:32]
    for t in (1, 3):
        want, _ = tvmc.metropolis(c.oans, th[t], sig0[t][ids], seed, t, 0, 2, chain_ids=ids)
        assert np.array_equal(sig[t][ids], want)
    dW = synth.random_normals(83, (T, c.nops), np.sqrt(dt))
    dW_d = torch.from_numpy(dW).cuda()
    E = torch.zeros((T, ns, 2), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(E)
    check(abi.otvmc_local_estimators(c.ans.handle, th_d, sp, T, ns, dW_d, dt, MIXED, E, v, None, work, nb))
    vv = from_dev_complex(v)[..., 0]
    w = tvmc.mc_weights(ns)
    t = 2
    terms = tvmc.local_terms(c.omodel, c.oans, th[t], sig[t])
    lpl = tvmc.expectation(w, terms["LpLd"]).real
    want_v = -1j * dt * tvmc.effective_energy(terms, lpl) + terms["B"] @ dW[t]
    assert rel_err(vv[t], want_v) < 1e-5
    G = torch.zeros((T, c.P, c.P), dtype=torch.float32, device="cuda")
    ob = torch.zeros((T, c.P), dtype=torch.float64, device="cuda")
    D = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    check(abi.otvmc_build_S_F(c.ans.handle, None, sp, v, T, ns, MIXED, None, G, ob, D, work, nb))
    delta = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    del work
    work, nb = c.work(T, ns, MIXED)
    check(abi.otvmc_solve_step(c.ans.handle, T, ns, MIXED, abi.OTVMC_REG_SHIFT, eps, 4.0, None, G, ob, D, delta,
                               None, work, nb))
    check(abi.otvmc_check(work))
    Gt, obt, Dt = G[t].cpu().numpy().astype(np.float64), ob[t].cpu().numpy(), from_dev_complex(D)[t, :, 0]
    # O columns from the spins (sites, then pairs j < k in row-major order)
    s = sig[t].astype(np.float64)
    pairs = c.oans.pairs
    rng = np.random.default_rng(5)
    ks = np.unique(np.concatenate([rng.integers(0, c.P, 40), [0, c.n - 1, c.n, c.P - 58, c.P - 1]]))

    def col(k):
        return s[:, k] if k < c.n else s[:, pairs[k - c.n, 0]] * s[:, pairs[k - c.n, 1]]

    vc = vv[t] - vv[t].mean()
    for i in ks:
        oi = col(i)
        assert obt[i] == oi.mean()
        assert abs(Dt[i] - (oi * vc).mean()) <= 1e-9 * np.abs(Dt).max()
        for j in ks[ks >= i]:
            assert Gt[i, j] == float(oi @ col(j))
    Gs = np.triu(Gt) + np.triu(Gt, 1).T
    A = Gs / ns - np.outer(obt, obt) + eps * np.eye(c.P)
    want_delta = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A, lower=True), Dt)
    assert rel_err(from_dev_complex(delta)[t, :, 0], want_delta) < 1e-4
