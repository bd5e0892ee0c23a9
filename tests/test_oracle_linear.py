"""Pins of the oracle's linear stochastic Schroedinger equation (App. B): the exact-state linear
SSE (Stratonovich form and Ito form) against the exact Lindblad solution, the otVMC force identity F^lin = F - i sum_n <L_n + L_n^+> N^n, the normalisation Q against the norm
of the exact-state trajectory where the ansatz is exact, and the Q-weighted MC ensemble against
Lindblad.  CPU only."""
import numpy as np
import pytest

from oracle import tvmc, lindblad, trajectories as tr
from oracle.ansatz import Jastrow
from oracle.model import Model, couplings, dense_hamiltonian, dense_jump_ops, coherent_x_state
from oracle.observables import ensemble_weighted, moments_from_rho
import synth


def _rho_moments(model, n, t):
    psi = coherent_x_state(n)
    rho, _ = lindblad.evolve(np.outer(psi, psi.conj()), dense_hamiltonian(model), dense_jump_ops(model), t, 1e-3)
    return moments_from_rho(rho, n)


def test_force_identity_of_the_linear_sse():
    """F^lin from the linear local effective energy equals F - i sum <L+L^+> N^n, so D^lin = D -
    dt sum <L+L^+> N^n (decay and dephasing, random parameters and samples)."""
    n = 5
    model = Model(J=couplings((n,), 1.0, 1.5), h=0.7, kappa=np.array([0.1, 0.2, 0.0, 0.3, 0.1]),
                  gamma=np.array([0.05, 0.0, 0.1, 0.0, 0.02]))
    ans = Jastrow(n)
    th = synth.random_theta(3, 1, ans.P, 0.3)[0]
    sig = synth.random_spins(4, 1, 200, n)[0]
    w = tvmc.mc_weights(200)
    dt = 0.01
    dW = synth.random_normals(5, (model.n_ops,), np.sqrt(dt))
    nl = tvmc.evaluate(model, ans, th, sig, w, dW, dt)
    li = tvmc.evaluate(model, ans, th, sig, w, dW, dt, linear=True)
    want = nl["F"] - 1j * nl["N"] @ nl["lpl"]
    assert np.abs(li["F"] - want).max() < 1e-12 * np.abs(want).max()
    assert np.abs(li["D"] - (nl["D"] - dt * nl["N"] @ nl["lpl"])).max() < 1e-13


@pytest.mark.parametrize("scheme", ["heun", "midpoint"])
def test_linear_sse_trajectory_average_converges_to_lindblad(scheme):
    """Eq. 3 with unnormalised expectations (the normalised moments weighted by <psi|psi>):
    within 4 standard errors of the exact solution, for the Stratonovich schemes and for the
    Ito equation by Euler-Maruyama; the mean norm stays 1 (trace preservation)."""
    n = 3
    m = Model(J=couplings((n,), 1.0, 1.5), h=0.6, kappa=0.4, gamma=0.1)
    dt, steps, nt = 0.01, 40, 400
    mom, _ = _rho_moments(m, n, dt * steps)
    for ito in (False, True):
        nrm = []
        mt, qt = tr.run_sse(m, nt, steps, dt, seed=5, scheme=scheme, ito=ito, linear=True, norm_out=nrm)
        Q = nrm[0][-1]
        M, _, dM = ensemble_weighted(mt[-1], qt[-1], Q)
        assert np.all(np.abs(M - mom) < 4 * dM + 3e-3), (ito, M, mom, dM)
        assert abs(Q.mean() - 1.0) < 4 * Q.std(ddof=1) / np.sqrt(nt) + 3e-3


def test_normalisation_follows_the_exact_norm_where_the_ansatz_is_exact():
    """h = 0 with local dephasing: the exact linear-SSE trajectory keeps the Jastrow form (its norm
    changes by the factor exp(sum_n Re(c_n) ...)), so enumeration otVMC of the linear SSE must
    follow it: normalised moments and Q = exp(ln Q) against <psi|psi> of the exact trajectory
    on the same noise, converging as dt -> 0."""
    n = 4
    model = Model(J=couplings((n,), 1.0, 1.5), h=0.0, kappa=0.0, gamma=0.1)
    ans = Jastrow(n)
    errs = []
    for dt in (0.01, 0.005, 0.0025):
        steps = int(round(0.1 / dt))
        lq, nr = [], []
        _, M1, Q1 = tr.run_enumeration(model, ans, 2, steps, dt, 11, "heun", eps=1e-12, linear=True, lnq_out=lq)
        M2, Q2 = tr.run_sse(model, 2, steps, dt, 11, "heun", linear=True, norm_out=nr)
        errs.append(max(np.abs(M1 - M2).max(), np.abs(np.exp(lq[0]) - nr[0]).max()))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 5e-4


def test_mc_linear_otvmc_ensemble_within_4_sigma_of_lindblad():
    """MC otVMC of the linear SSE with the Q-weighted average (the expectation-linear formula of
    App. B), 4 spins with decay, against the exact solution at t = 0.2."""
    n = 4
    model = Model(J=couplings((n,), 1.0, 1.5), h=1.0, kappa=0.1, gamma=0.0)
    ans = Jastrow(n)
    dt, steps, nt, ns = 0.02, 10, 48, 512
    lq = []
    _, _, m, q = tr.run_mc(model, ans, nt, ns, steps, dt, seed=21, scheme="heun", eps=1e-4, linear=True,
                           lnq_out=lq)
    mom, _ = _rho_moments(model, n, dt * steps)
    M, C, dM = ensemble_weighted(m[-1], q[-1], np.exp(lq[0][-1]))
    assert np.all(np.abs(M - mom) <= 4 * dM + 2e-3), (M, mom, dM)
