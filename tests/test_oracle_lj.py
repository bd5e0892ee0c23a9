"""Pins of the oracle's partially inhomogeneous long-range Jastrow ansaetze LJPHd and LJH (Eq. 12
and the paragraph after it): parameter counts, the full Jastrow as the fully inhomogeneous
limit, log-derivatives and flip ratios against brute force, local estimators against dense
operators, and exactness of the homogeneous ansatz for the unitary Ising chain whose couplings
depend only on the distance.  CPU only."""
import numpy as np
import pytest

from oracle import tvmc, trajectories as tr
from oracle.ansatz import Jastrow, lj_ansatz, lj_groups
from oracle.model import Model, couplings, dense_hamiltonian, dense_jump_ops, spins_of_index
import synth


def _theta(ans, seed, scale=0.3):
    return synth.random_theta(seed, 1, ans.P, scale)[0]


@pytest.mark.parametrize("n", [5, 10, 11])
def test_parameter_counts(n):
    """Open chain: N biases, the N - D pairs of each distance D <= d free, one parameter per
    distance D > d: P = 2N - 1 - d + N d - d(d+1)/2.  At d = 0 (LJH) and d = N - 1 (LJNH) this
    is the paper's count 2N - 1 - d + N d / 2.  Periodic chain (nearest-image distance, at most
    N // 2): N pairs at each distance below N / 2 and N / 2 pairs at N / 2."""
    for d in range(n):
        P = n + len(lj_groups(n, d, pbc=False))
        assert P == 2 * n - 1 - d + n * d - d * (d + 1) // 2
        if d in (0, n - 1):
            assert 2 * P == 2 * (2 * n - 1 - d) + n * d
    for d in range(n // 2 + 1):
        P = n + len(lj_groups(n, d, pbc=True))
        free = sum(n if 2 * D < n else n // 2 for D in range(1, d + 1))
        assert P == n + free + (n // 2 - d)
    # every pair belongs to exactly one group
    for pbc in (False, True):
        g = lj_groups(n, 1, pbc)
        flat = [p for grp in g for p in grp]
        assert sorted(flat) == [(j, k) for j in range(n) for k in range(j + 1, n)]


def test_fully_inhomogeneous_limit_is_the_full_jastrow():
    n = 6
    lj, full = lj_ansatz(n, n - 1), Jastrow(n)
    assert lj.P == full.P
    th = _theta(full, 1)
    sig = synth.random_spins(2, 1, 40, n)[0]
    assert np.array_equal(lj.O(th, sig), full.O(th, sig))
    assert np.allclose(lj.logpsi(th, sig), full.logpsi(th, sig), rtol=0, atol=1e-14)
    assert np.allclose(lj.log_flip_ratios(th, sig), full.log_flip_ratios(th, sig), rtol=0, atol=1e-14)


@pytest.mark.parametrize("d,pbc", [(1, False), (0, True), (2, True), (0, False)])
def test_flip_ratios_and_log_derivatives(d, pbc):
    n = 7
    ans = lj_ansatz(n, d, pbc)
    th = _theta(ans, 3)
    sig = synth.random_spins(4, 1, 25, n)[0]
    lr = ans.log_flip_ratios(th, sig)
    l2 = ans.log_pair_flip_ratios(th, sig)
    for j in range(n):
        f = sig.copy()
        f[:, j] *= -1
        want = np.exp(ans.logpsi(th, f) - ans.logpsi(th, sig))
        assert (np.abs(np.exp(lr[:, j]) - want) / np.maximum(1.0, np.abs(want))).max() < 1e-12
        for k in range(n):
            if k != j:
                f2 = sig.copy()
                f2[:, [j, k]] *= -1
                dd = ans.logpsi(th, f2) - ans.logpsi(th, sig)
                want = np.exp(dd)
                assert (np.abs(np.exp(l2[:, j, k]) - want) / np.maximum(1.0, np.abs(want))).max() < 1e-12
    O = ans.O(th, sig)
    h = 1e-6
    for k in range(ans.P):
        e = np.zeros(ans.P)
        e[k] = h
        fd = (ans.logpsi(th + e, sig) - ans.logpsi(th - e, sig)) / (2 * h)
        fdi = (ans.logpsi(th + 1j * e, sig) - ans.logpsi(th - 1j * e, sig)) / (2j * h)
        assert np.abs(fd - O[:, k]).max() < 1e-7 and np.abs(fdi - O[:, k]).max() < 1e-7
    site = np.arange(25) % n
    assert np.allclose(tvmc.log_flip_ratio_at(ans, th, sig, site), lr[np.arange(25), site])


def test_local_estimators_match_dense_operators():
    n = 5
    ans = lj_ansatz(n, 1)
    model = Model(J=couplings((n,), 1.0, 1.5), h=0.7, kappa=np.array([0.1, 0.2, 0.0, 0.3, 0.1]),
                  gamma=np.array([0.05, 0.0, 0.1, 0.0, 0.02]))
    th = _theta(ans, 5)
    sig = spins_of_index(n)
    psi = np.exp(ans.logpsi(th, sig))
    H, Ls = dense_hamiltonian(model), dense_jump_ops(model)
    p = np.abs(psi) ** 2
    p /= p.sum()
    lpl = np.array([np.sum(p * (((L + L.conj().T) @ psi) / psi)).real for L in Ls])
    Heff = H.astype(complex)
    for L, m in zip(Ls, lpl):
        Heff = Heff - 0.5j * (L.conj().T @ L - 2 * m * L + L @ L)
    terms = tvmc.local_terms(model, ans, th, sig)
    lo = tvmc.expectation(p, terms["LpLd"]).real
    assert np.allclose(lo, lpl, atol=1e-12)
    assert np.abs(tvmc.effective_energy(terms, lo) - (Heff @ psi) / psi).max() < 1e-10


@pytest.mark.parametrize("pbc", [False, True])
def test_homogeneous_ansatz_is_exact_for_the_unitary_ising_chain(pbc):
    """gamma = 0, h = 0, couplings J/r^alpha that depend only on the (open or nearest-image)
    distance: the state exp(-i t sum J_jk s_j s_k) from +x is an LJH state with eta_D = -i t J_D,
    so enumeration tVMC with LJH must follow it to integrator error (and <s^x_j> =
    prod_k cos(2 J_jk t))."""
    n = 6
    J = couplings((n,), 1.0, 1.5, pbc=pbc)
    model = Model(J=J, h=0.0, kappa=0.0, gamma=0.0)
    ans = lj_ansatz(n, 0, pbc)
    assert ans.P < Jastrow(n).P
    dt, steps = 0.01, 15
    th, M, Q = tr.run_enumeration(model, ans, 1, steps, dt, 3, "heun", eps=1e-12)
    a, eta = ans.split(th[0])
    assert np.abs(eta + 1j * dt * steps * J).max() < 1e-10
    assert np.abs(a).max() < 1e-12
    t = dt * steps
    sx = [np.prod([np.cos(2 * J[j, k] * t) for k in range(n) if k != j]) for j in range(n)]
    assert abs(M[-1, 0, 0] - np.mean(sx)) < 1e-10


def test_homogeneous_ansatz_with_dephasing_converges_to_exact_sse():
    """h = 0 with local dephasing: the exact trajectory multiplies the state by site-dependent
    factors exp(c_j s_j), which the inhomogeneous biases of LJH absorb, and keeps
    eta = -i t J; LJH tVMC therefore converges to the exact-state trajectory as dt -> 0."""
    n = 4
    model = Model(J=couplings((n,), 1.0, 1.5), h=0.0, kappa=0.0, gamma=0.1)
    ans = lj_ansatz(n, 0)
    errs = []
    for dt in (0.01, 0.005, 0.0025):
        steps = int(round(0.1 / dt))
        _, M1, Q1 = tr.run_enumeration(model, ans, 1, steps, dt, 11, "heun", eps=1e-12)
        M2, Q2 = tr.run_sse(model, 1, steps, dt, 11, "heun")
        errs.append(max(np.abs(M1 - M2).max(), np.abs(Q1 - Q2).max()))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 5e-4
