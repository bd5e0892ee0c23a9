"""Pins of the oracle's otVMC part: ansaetze, local estimators, S/F/N/D, solves, sampler,
observables and trajectory ensembles.  CPU only."""
import numpy as np
import pytest
import scipy.stats

from oracle import tvmc, philox, lindblad, trajectories as tr
from oracle.ansatz import Jastrow, RBM, log2cosh
from oracle.model import (Model, couplings, dense_hamiltonian, dense_jump_ops, coherent_x_state,
                          spins_of_index, pauli_ops)
from oracle.observables import moments_from_samples, moments_from_state, squeezing, ensemble, moments_from_rho
import synth


def _theta(ans, seed, scale=0.3):
    return synth.random_theta(seed, 1, ans.P, scale)[0]


def _psi_vector(ans, theta):
    sig = spins_of_index(ans.n)
    return np.exp(ans.logpsi(theta, sig)), sig


@pytest.mark.parametrize("ans", [Jastrow(5), RBM(4, 3)])
def test_flip_ratios_match_brute_force(ans):
    th = _theta(ans, 1)
    sig = synth.random_spins(2, 1, 30, ans.n)[0]
    lr = ans.log_flip_ratios(th, sig)
    for j in range(ans.n):
        f = sig.copy()
        f[:, j] *= -1
        d = ans.logpsi(th, f) - ans.logpsi(th, sig)
        assert np.abs(np.exp(lr[:, j]) - np.exp(d)).max() < 1e-12
    l2 = ans.log_pair_flip_ratios(th, sig)
    for j in range(ans.n):
        for k in range(ans.n):
            if j == k:
                continue
            f = sig.copy()
            f[:, [j, k]] *= -1
            d = ans.logpsi(th, f) - ans.logpsi(th, sig)
            assert np.abs(np.exp(l2[:, j, k]) - np.exp(d)).max() < 1e-12
    site = np.arange(30) % ans.n
    assert np.allclose(tvmc.log_flip_ratio_at(ans, th, sig, site), lr[np.arange(30), site])


@pytest.mark.parametrize("ans", [Jastrow(4), RBM(3, 2)])
def test_log_derivatives_match_finite_differences(ans):
    th = _theta(ans, 3)
    sig = synth.random_spins(4, 1, 10, ans.n)[0]
    O = ans.O(th, sig)
    h = 1e-6
    for k in range(ans.P):
        e = np.zeros(ans.P)
        e[k] = h
        # holomorphic ansatz: d/dtheta along the real axis
        fd = (ans.logpsi(th + e, sig) - ans.logpsi(th - e, sig)) / (2 * h)
        assert np.abs(fd - O[:, k]).max() < 1e-8
        fdi = (ans.logpsi(th + 1j * e, sig) - ans.logpsi(th - 1j * e, sig)) / (2j * h)
        assert np.abs(fdi - O[:, k]).max() < 1e-8


def test_log2cosh_stable():
    z = np.array([0.3 + 0.2j, -800 + 1j, 800 - 2j, 1e-3j])
    ref = np.log(2 * np.cosh(z[[0, 3]]))
    assert np.allclose(log2cosh(z[[0, 3]]), ref)
    assert np.isfinite(log2cosh(z)).all()


def _dense_local(model, ans, theta):
    """<x|A|psi>/psi(x) from dense operators, with exact <L+L^+>."""
    psi, sig = _psi_vector(ans, theta)
    H = dense_hamiltonian(model)
    Ls = dense_jump_ops(model)
    p = np.abs(psi) ** 2
    p /= p.sum()
    lpl = np.array([np.sum(p * (((L + L.conj().T) @ psi) / psi)).real for L in Ls])
    Heff = H.astype(complex)
    for L, m in zip(Ls, lpl):
        Heff = Heff - 0.5j * (L.conj().T @ L - 2 * m * L + L @ L)
    E = (Heff @ psi) / psi
    B = np.stack([(L @ psi) / psi for L in Ls], axis=1)
    return E, B, lpl, sig, p


@pytest.mark.parametrize("ans", [Jastrow(4), RBM(4, 2)])
def test_local_estimators_match_dense_operators(ans):
    n = ans.n
    model = Model(J=couplings((n,), 1.0, 1.5), h=0.7, kappa=np.array([0.1, 0.2, 0.0, 0.3]),
                  gamma=np.array([0.05, 0.0, 0.1, 0.0]))
    th = _theta(ans, 5)
    E, B, lpl, sig, p = _dense_local(model, ans, th)
    terms = tvmc.local_terms(model, ans, th, sig)
    lpl_o = tvmc.expectation(p, terms["LpLd"]).real
    assert np.allclose(lpl_o, lpl, atol=1e-12)
    Eo = tvmc.effective_energy(terms, lpl_o)
    assert np.abs(Eo - E).max() < 1e-10
    assert np.abs(terms["B"] - B).max() < 1e-12


def test_covariances_hermitian_psd_and_d_assembly():
    ans = Jastrow(5)
    model = Model(J=couplings((5,), 1.0, 1.5), h=1.0, kappa=0.1, gamma=0.05)
    th = _theta(ans, 7, 0.1)
    sig = synth.random_spins(8, 1, 200, 5)[0]
    w = tvmc.mc_weights(200)
    dW = synth.random_normals(9, model.n_ops, 0.1)
    ev = tvmc.evaluate(model, ans, th, sig, w, dW, 0.01)
    S = ev["S"]
    assert np.abs(S - S.conj().T).max() < 1e-14
    assert np.linalg.eigvalsh(S).min() > -1e-12
    # D = Cov(O^*, v) with v = -i dt E_eff + sum_n dW_n B^n (linearity of the covariance)
    v = tvmc.local_v(ev, dW, 0.01)
    assert np.abs(tvmc.covariance(w, ev["O"], v[:, None])[:, 0] - ev["D"]).max() < 1e-13


def test_mc_covariances_converge_to_exact():
    ans = Jastrow(4)
    model = Model(J=couplings((4,), 1.0, 1.5), h=1.0, kappa=0.1, gamma=0.0)
    th = _theta(ans, 11, 0.2)
    dW = np.zeros(model.n_ops)
    ex = tvmc.evaluate_enumeration(model, ans, th, dW, 1.0)
    sig = tvmc.all_configs(4)
    p = tvmc.exact_weights(ans, th, sig)
    idx = np.random.default_rng(0).choice(len(p), size=400000, p=p)
    mc = tvmc.evaluate(model, ans, th, sig[idx], tvmc.mc_weights(len(idx)), dW, 1.0)
    assert np.abs(mc["S"] - ex["S"]).max() < 0.01
    assert np.abs(mc["F"] - ex["F"]).max() < 0.03


def test_shift_solve_residual_and_snr_limit():
    g = np.random.default_rng(1)
    ns, P = 300, 12
    O = g.normal(size=(ns, P)) + 1j * g.normal(size=(ns, P))
    v = g.normal(size=ns) + 1j * g.normal(size=ns)
    w = tvmc.mc_weights(ns)
    S = tvmc.covariance(w, O, O)
    D = tvmc.covariance(w, O, v[:, None])[:, 0]
    x = tvmc.solve_shift(S, D, 1e-3)
    assert np.abs((S + 1e-3 * np.eye(P)) @ x - D).max() < 1e-12
    # SNR filter with vanishing thresholds is the plain pseudo-inverse
    y = tvmc.solve_snr(S, D, O, v, w, snr_thresh=1e-12, eps_svd=1e-300)
    assert np.abs(y - np.linalg.pinv(S) @ D).max() < 1e-10


@pytest.mark.parametrize("ns,P,mc", [(40, 90, True), (120, 30, True), (64, 200, False)])
def test_push_through_solve_equals_shift_solve(ns, P, mc):
    """The Ns x Ns form of the diagonal-shift solve gives the P x P solve's delta, with P above
    and below Ns and with non-uniform (exact-expectation) weights."""
    g = np.random.default_rng(ns + P)
    O = g.normal(size=(ns, P)) + 1j * g.normal(size=(ns, P))
    v = g.normal(size=ns) + 1j * g.normal(size=ns)
    w = tvmc.mc_weights(ns) if mc else g.random(ns)
    w = w / w.sum()
    eps = 1e-3
    S = tvmc.covariance(w, O, O)
    D = tvmc.covariance(w, O, v[:, None])[:, 0]
    want = tvmc.solve_shift(S, D, eps)
    got = tvmc.solve_shift_push(O, v, w, eps)
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()
    # and it solves the P x P system
    assert np.abs((S + eps * np.eye(P)) @ got - D).max() < 1e-10 * np.abs(D).max()


def test_enumeration_tvmc_unitary_ising_is_exact():
    """gamma = 0, h = 0: psi(t) is the Jastrow state eta = -i t J, a = 0."""
    n = 5
    J = couplings((n,), 1.0, 1.5)
    model = Model(J=J, h=0.0, kappa=0.0, gamma=0.0)
    ans = Jastrow(n)
    dt, steps = 0.01, 15
    for scheme in ("heun", "midpoint"):
        th, M, Q = tr.run_enumeration(model, ans, 1, steps, dt, 3, scheme, eps=1e-12)
        a, eta = ans.split(th[0])
        assert np.abs(eta + 1j * dt * steps * J).max() < 1e-10
        assert np.abs(a).max() < 1e-12
        t = dt * steps
        sx = [np.prod([np.cos(2 * J[j, k] * t) for k in range(n) if k != j]) for j in range(n)]
        assert abs(M[-1, 0, 0] - np.mean(sx)) < 1e-10


def test_enumeration_tvmc_dephasing_converges_to_exact_sse():
    """h = 0 with dephasing only: the exact trajectory stays a Jastrow state, so the
    variational and the exact-state trajectories agree up to the integrator error."""
    n = 4
    model = Model(J=couplings((n,), 1.0, 1.5), h=0.0, kappa=0.0, gamma=0.1)
    ans = Jastrow(n)
    errs = []
    for dt in (0.01, 0.005, 0.0025):
        steps = int(round(0.1 / dt))
        _, M1, Q1 = tr.run_enumeration(model, ans, 1, steps, dt, 11, "heun", eps=1e-12)
        M2, Q2 = tr.run_sse(model, 1, steps, dt, 11, "heun")
        errs.append(max(np.abs(M1 - M2).max(), np.abs(Q1 - Q2).max()))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 5e-4


def test_metropolis_samples_psi_squared():
    n = 4
    ans = Jastrow(n)
    th = _theta(ans, 13, 0.2)
    sig0 = philox.initial_spins(5, 0, 4000, n)
    sig, acc = tvmc.metropolis(ans, th, sig0, 5, 0, 0, n_sweep=30)
    idx = ((sig > 0).astype(int) << np.arange(n)).sum(axis=1)
    counts = np.bincount(idx, minlength=2 ** n)
    p = tvmc.exact_weights(ans, th, tvmc.all_configs(n))
    chi2 = scipy.stats.chisquare(counts, p * counts.sum())
    assert chi2.pvalue > 1e-3
    assert acc.mean() > 0


def test_metropolis_samples_rbm_psi_squared():
    """The RBM branch of the proposal ratios (log 2cosh differences of the hidden angles):
    chains of a complex RBM (4 sites, 3 hidden units) visit the 16 configurations with the
    frequencies |psi|^2 / Z computed by enumeration."""
    n, m = 4, 3
    ans = RBM(n, m)
    th = _theta(ans, 29, 0.4)
    sig0 = philox.initial_spins(7, 0, 4000, n)
    sig, acc = tvmc.metropolis(ans, th, sig0, 7, 0, 0, n_sweep=30)
    idx = ((sig > 0).astype(int) << np.arange(n)).sum(axis=1)
    counts = np.bincount(idx, minlength=2 ** n)
    p = tvmc.exact_weights(ans, th, tvmc.all_configs(n))
    assert p.max() / p.min() > 1.5  # not the uniform distribution
    chi2 = scipy.stats.chisquare(counts, p * counts.sum())
    assert chi2.pvalue > 1e-3
    assert acc.mean() > 0


def test_ensemble_moments_and_standard_error_closed_form():
    """Eq. 3 averages on hand-made trajectories: M the mean, C = <q> - M M^T, and dM the sample
    standard deviation (ddof 1) over sqrt(N_T); for q = m m^T (product states) C is the
    population covariance of the m's."""
    m = np.array([[1.0, 0.0, 0.5], [-1.0, 0.0, 0.5], [1.0, 0.0, -0.5], [-1.0, 0.0, -0.5]])
    q = np.einsum("ta,tb->tab", m, m)
    M, C, dM = ensemble(m, q)
    assert np.allclose(M, 0.0)
    assert np.allclose(dM, [np.sqrt(4.0 / 3.0) / 2.0, 0.0, np.sqrt(1.0 / 3.0) / 2.0])
    assert np.allclose(C, np.cov(m.T, bias=True))
    assert np.allclose(np.diag(C), [1.0, 0.0, 0.25])


def test_metropolis_chain_is_deterministic_and_counter_based():
    ans = Jastrow(6)
    th = _theta(ans, 2, 0.2)
    sig0 = philox.initial_spins(1, 4, 64, 6)
    a, _ = tvmc.metropolis(ans, th, sig0, 1, 4, 3, 2)
    b, _ = tvmc.metropolis(ans, th, sig0, 1, 4, 3, 2)
    c, _ = tvmc.metropolis(ans, th, sig0, 1, 4, 4, 2)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_observables_coherent_state_and_exact_weights():
    n = 6
    ans = Jastrow(n)
    sig = tvmc.all_configs(n)
    th = np.zeros(ans.P, complex)
    m, q = moments_from_samples(ans, th, sig, tvmc.exact_weights(ans, th, sig))
    C = q - np.outer(m, m)
    assert np.allclose(m, [1, 0, 0], atol=1e-14)
    assert np.allclose(C[1:, 1:], np.eye(2) / n, atol=1e-14)
    assert abs(squeezing(m, C, n) - 1) < 1e-12
    # generic state: local estimators under exact weights equal the dense expectations
    for a in (Jastrow(4), RBM(4, 3)):
        th = _theta(a, 17, 0.3)
        psi, s = _psi_vector(a, th)
        m1, q1 = moments_from_samples(a, th, s, tvmc.exact_weights(a, th, s))
        m2, q2 = moments_from_state(psi, a.n)
        assert np.abs(m1 - m2).max() < 1e-12 and np.abs(q1 - q2).max() < 1e-12


def test_squeezing_of_known_covariance():
    M = np.array([0.0, 0.0, 0.8])
    C = np.diag([0.02, 0.05, 0.0])
    assert abs(squeezing(M, C, 10) - 10 * 0.02 / 0.64) < 1e-14


@pytest.mark.slow
def test_mc_otvmc_ensemble_within_3_sigma_of_lindblad():
    n = 4
    model = Model(J=couplings((n,), 1.0, 1.5), h=1.0, kappa=0.1, gamma=0.0)
    ans = Jastrow(n)
    dt, steps, nt, ns = 0.02, 10, 24, 512
    th, sig, m, q = tr.run_mc(model, ans, nt, ns, steps, dt, seed=21, scheme="heun", eps=1e-4)
    psi = coherent_x_state(n)
    rho, _ = lindblad.evolve(np.outer(psi, psi.conj()), dense_hamiltonian(model), dense_jump_ops(model),
                             dt * steps, 1e-3)
    mom, _ = moments_from_rho(rho, n)
    M, C, dM = ensemble(m[-1], q[-1])
    assert np.all(np.abs(M - mom) <= 3 * dM + 1e-3)
