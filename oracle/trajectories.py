"""Trajectory ensembles: MC otVMC, enumeration otVMC and exact-state SSE (Eq. 3, App. C).

Test infrastructure (oracle side).  All three use the same Wiener increments, drawn by the
counter-based generator of oracle.philox from (seed, trajectory, step), so that a given
trajectory sees the same noise path in every method.

Measurement convention: the moments at time t_i = i dt are taken from the configurations
drawn at theta_i (the predictor-stage samples of step i); after the last step one more
sampling pass (evaluation index 2 n_steps) gives the moments at the final time.
"""
import numpy as np

from . import philox, tvmc, sse
from .observables import moments_from_samples, moments_from_state
from .model import dense_hamiltonian, dense_jump_ops, coherent_x_state


def run_mc(model, ans, ntraj, ns, n_steps, dt, seed, scheme="heun", n_sweep=2, eps=1e-4,
           traj0=0, theta0=None, measure=True, reg="shift", push=False):
    """MC otVMC; returns theta (ntraj, P), spins, moments m (n_meas, ntraj, 3), q (.., 3, 3).

    push=True solves the diagonal-shift system through its Ns x Ns form (tvmc.solve_shift_push,
    the same delta) and never forms S: for parameter counts far above Ns.
    """
    P, n = ans.P, ans.n
    n_ops = model.n_ops
    thetas, sigs, ms, qs = [], [], [], []
    w = tvmc.mc_weights(ns)
    for t in range(ntraj):
        tid = traj0 + t
        theta = np.zeros(P, complex) if theta0 is None else np.array(theta0, complex)
        sig = philox.initial_spins(seed, tid, ns, n)
        m_t, q_t = [], []
        for i in range(n_steps):
            dW = philox.wiener_increments(seed, [tid], i, n_ops, dt)[0]

            def increment(th, stage):
                nonlocal sig
                sig, _ = tvmc.metropolis(ans, th, sig, seed, tid, 2 * i + stage, n_sweep)
                if stage == 0 and measure:
                    m, q = moments_from_samples(ans, th, sig, w)
                    m_t.append(m)
                    q_t.append(q)
                ev = tvmc.evaluate(model, ans, th, sig, w, dW, dt, with_S=not push)
                if reg == "shift" and push:
                    return tvmc.solve_shift_push(ev["O"], tvmc.local_v(ev, dW, dt), w, eps)
                if reg == "shift":
                    return tvmc.solve_shift(ev["S"], ev["D"], eps)
                return tvmc.solve_snr(ev["S"], ev["D"], ev["O"], tvmc.local_v(ev, dW, dt), w)

            theta, _, _ = tvmc.sde_step(theta, increment, scheme)
        if measure:
            sig, _ = tvmc.metropolis(ans, theta, sig, seed, tid, 2 * n_steps, n_sweep)
            m, q = moments_from_samples(ans, theta, sig, w)
            m_t.append(m)
            q_t.append(q)
        thetas.append(theta)
        sigs.append(sig)
        ms.append(m_t)
        qs.append(q_t)
    m = np.array(ms).transpose(1, 0, 2) if measure else None
    q = np.array(qs).transpose(1, 0, 2, 3) if measure else None
    return np.array(thetas), np.array(sigs), m, q


def run_enumeration(model, ans, ntraj, n_steps, dt, seed, scheme="heun", eps=1e-10, traj0=0):
    """Enumeration otVMC (exact expectations): per-step moments (n_steps+1, ntraj, ...)."""
    from .tvmc import all_configs, exact_weights
    P, n = ans.P, ans.n
    sig = all_configs(n)
    ms, qs, thetas = [], [], []
    for t in range(ntraj):
        tid = traj0 + t
        theta = np.zeros(P, complex)
        m_t, q_t = [], []
        for i in range(n_steps):
            w = exact_weights(ans, theta, sig)
            m, q = moments_from_samples(ans, theta, sig, w)
            m_t.append(m)
            q_t.append(q)
            dW = philox.wiener_increments(seed, [tid], i, model.n_ops, dt)[0]

            def increment(th, stage):
                ev = tvmc.evaluate_enumeration(model, ans, th, dW, dt)
                return tvmc.solve_shift(ev["S"], ev["D"], eps)

            theta, _, _ = tvmc.sde_step(theta, increment, scheme)
        w = exact_weights(ans, theta, sig)
        m, q = moments_from_samples(ans, theta, sig, w)
        m_t.append(m)
        q_t.append(q)
        ms.append(m_t)
        qs.append(q_t)
        thetas.append(theta)
    return np.array(thetas), np.array(ms).transpose(1, 0, 2), np.array(qs).transpose(1, 0, 2, 3)


def run_sse(model, ntraj, n_steps, dt, seed, scheme="heun", traj0=0, ito=False):
    """Exact-state trajectories of Eq. 4 (or Eq. 2 by Euler-Maruyama when ito=True)."""
    n = model.n
    H = dense_hamiltonian(model)
    Ls = dense_jump_ops(model)
    ms, qs = [], []
    for t in range(ntraj):
        tid = traj0 + t
        psi = coherent_x_state(n)
        m_t, q_t = [], []
        for i in range(n_steps):
            m, q = moments_from_state(psi, n)
            m_t.append(m)
            q_t.append(q)
            dW = philox.wiener_increments(seed, [tid], i, model.n_ops, dt)[0]
            if ito:
                psi = sse.step_ito_em(psi, H, Ls, dt, dW)
            else:
                psi = sse.step_strat(psi, H, Ls, dt, dW, scheme)
        m, q = moments_from_state(psi, n)
        m_t.append(m)
        q_t.append(q)
        ms.append(m_t)
        qs.append(q_t)
    return np.array(ms).transpose(1, 0, 2), np.array(qs).transpose(1, 0, 2, 3)
