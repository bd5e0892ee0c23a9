"""Pins of the oracle's exact references: Philox, Lindblad integration, exact-state SSE,
and the closed form of App. D.  CPU only."""
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

from oracle import philox, lindblad, sse, fossfeig
from oracle.model import (Model, couplings, dense_hamiltonian, dense_jump_ops, coherent_x_state,
                          pauli_ops, spins_of_index)
from oracle.observables import moments_from_rho, moments_from_state
from oracle import trajectories as tr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_wiener_increments_are_gaussian_with_variance_dt():
    dt = 0.01
    z = philox.wiener_increments(123, np.arange(2000), 5, 7, dt).ravel()
    assert scipy.stats.kstest(z / np.sqrt(dt), "norm").pvalue > 1e-3
    # different steps / trajectories give different increments
    z2 = philox.wiener_increments(123, np.arange(2000), 6, 7, dt).ravel()
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.05


def test_initial_spins_uniform():
    s = philox.initial_spins(9, 3, 4096, 70)
    assert s.shape == (4096, 70)
    assert abs(s.mean()) < 0.02
    assert set(np.unique(s)) == {-1, 1}


def _rho0(n):
    psi = coherent_x_state(n)
    return np.outer(psi, psi.conj())


@pytest.mark.parametrize("n", [2, 3])
def test_lindblad_rk4_matches_expm_of_liouvillian(n):
    m = Model(J=couplings((n,), 0.7, 1.5), h=0.4, kappa=0.3, gamma=0.2)
    H, Ls = dense_hamiltonian(m), dense_jump_ops(m)
    t = 0.6
    rho, _ = lindblad.evolve(_rho0(n), H, Ls, t, 2e-3)
    vec = scipy.linalg.expm(lindblad.liouvillian(H, Ls) * t) @ _rho0(n).ravel()
    assert np.abs(rho.ravel() - vec).max() < 1e-9


def test_single_spin_decay_closed_form():
    m = Model(J=np.zeros((1, 1)), h=0.0, kappa=0.4, gamma=0.0)
    t = 1.3
    rho, _ = lindblad.evolve(_rho0(1), dense_hamiltonian(m), dense_jump_ops(m), t, 1e-3)
    mom, _ = moments_from_rho(rho, 1)
    assert abs(mom[2] - (np.exp(-0.4 * t) - 1)) < 1e-10
    assert abs(mom[0] - np.exp(-0.2 * t)) < 1e-10


def test_pure_dephasing_ising_closed_form():
    n = 4
    J = couplings((n,), 1.0, 1.5)
    g = 0.15
    m = Model(J=J, h=0.0, kappa=0.0, gamma=g)
    t = 0.8
    rho, _ = lindblad.evolve(_rho0(n), dense_hamiltonian(m), dense_jump_ops(m), t, 1e-3)
    for j in range(n):
        sx = pauli_ops(n, j)[0]
        expect = np.exp(-2 * g * t) * np.prod([np.cos(2 * J[j, k] * t) for k in range(n) if k != j])
        assert abs(np.trace(sx @ rho).real - expect) < 1e-9


def test_lindblad_invariants():
    n = 3
    m = Model(J=couplings((n,), 1.0, 1.0), h=0.8, kappa=0.5, gamma=0.1)
    rho, _ = lindblad.evolve(_rho0(n), dense_hamiltonian(m), dense_jump_ops(m), 1.0, 5e-3)
    assert abs(np.trace(rho) - 1) < 1e-12
    assert np.abs(rho - rho.conj().T).max() < 1e-12
    assert np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)).min() > -1e-10


@pytest.mark.parametrize("n,kappa,alpha", [(4, 0.5, 1.0), (5, 0.3, 1.0), (6, 0.2, 1.5)])
def test_fossfeig_matches_exact_lindblad(n, kappa, alpha):
    Jd = fossfeig.ring_couplings(n, 1.0, alpha, kac=True)
    Jij = np.array([[0.0 if i == j else Jd[(i - j) % n] for j in range(n)] for i in range(n)])
    m = Model(J=Jij, h=0.0, kappa=kappa, gamma=0.0)
    t = 0.9
    rho, _ = lindblad.evolve(_rho0(n), dense_hamiltonian(m), dense_jump_ops(m), t, 1e-3)
    mom, q = moments_from_rho(rho, n)
    C = q - np.outer(mom, mom)
    Mf, Cf = fossfeig.fossfeig(Jd, kappa, t)
    assert np.abs(mom - Mf).max() < 1e-9
    assert np.abs(C - Cf).max() < 1e-9
    assert abs(Mf[2] - (np.exp(-kappa * t) - 1)) < 1e-14
    # the LITF sign (J_ij = -J_d) flips only the y components
    m2 = Model(J=-Jij, h=0.0, kappa=kappa, gamma=0.0)
    rho2, _ = lindblad.evolve(_rho0(n), dense_hamiltonian(m2), dense_jump_ops(m2), t, 1e-3)
    mom2, _ = moments_from_rho(rho2, n)
    assert np.allclose(mom2, mom * np.array([1, -1, 1]), atol=1e-9)


def test_fossfeig_coherent_state_at_t0():
    Jd = fossfeig.ring_couplings(10, 1.0, 1.0)
    M, C = fossfeig.fossfeig(Jd, 0.5, 0.0)
    assert np.allclose(M, [1, 0, 0], atol=1e-14)
    assert np.allclose(np.diag(C), [0, 0.1, 0.1], atol=1e-14)


def test_sse_unitary_limit_is_schroedinger():
    n = 3
    m = Model(J=couplings((n,), 1.0, 1.5), h=0.7, kappa=0.0, gamma=0.0)
    H = dense_hamiltonian(m)
    psi = coherent_x_state(n)
    dt, steps = 1e-3, 300
    for _ in range(steps):
        psi = sse.step_strat(psi, H, [], dt, [], "midpoint")
    exact = scipy.linalg.expm(-1j * H * dt * steps) @ coherent_x_state(n)
    assert np.abs(psi - exact).max() < 1e-5


def test_sse_norm_drift_vanishes_with_dt():
    n = 3
    m = Model(J=couplings((n,), 1.0, 1.5), h=0.5, kappa=0.3, gamma=0.1)
    H, Ls = dense_hamiltonian(m), dense_jump_ops(m)
    drifts = []
    for dt in (4e-3, 1e-3):
        steps = int(0.4 / dt)
        psi = coherent_x_state(n)
        g = np.random.default_rng(0)
        for _ in range(steps):
            dW = g.normal(0, np.sqrt(dt), len(Ls))
            psi = sse.step_ito_em(psi, H, Ls, dt, dW)
        drifts.append(abs(np.vdot(psi, psi).real - 1))
    assert drifts[1] < drifts[0]
    assert drifts[1] < 0.05


@pytest.mark.parametrize("scheme", ["heun", "midpoint"])
def test_sse_trajectory_average_converges_to_lindblad(scheme):
    n = 3
    m = Model(J=couplings((n,), 1.0, 1.5), h=0.6, kappa=0.4, gamma=0.1)
    dt, steps, nt = 0.01, 40, 300
    mt, qt = tr.run_sse(m, nt, steps, dt, seed=5, scheme=scheme)
    rho, _ = lindblad.evolve(_rho0(n), dense_hamiltonian(m), dense_jump_ops(m), dt * steps, 1e-3)
    mom, q = moments_from_rho(rho, n)
    mean = mt[-1].mean(axis=0)
    err = mt[-1].std(axis=0, ddof=1) / np.sqrt(nt)
    assert np.all(np.abs(mean - mom) < 4 * err + 2e-3)
    # Ito Euler-Maruyama on Eq. 2 agrees as well
    mi, _ = tr.run_sse(m, nt, steps, dt, seed=5, ito=True)
    assert np.all(np.abs(mi[-1].mean(axis=0) - mom) < 4 * mi[-1].std(axis=0, ddof=1) / np.sqrt(nt) + 4e-3)
