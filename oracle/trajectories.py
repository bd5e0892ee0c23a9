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
           traj0=0, theta0=None, measure=True, reg="shift", push=False, linear=False, lnq_out=None):
    """MC otVMC; returns theta (ntraj, P), spins, moments m (n_meas, ntraj, 3), q (.., 3, 3).

    push=True solves the diagonal-shift system through its Ns x Ns form (tvmc.solve_shift_push,
    the same delta) and never forms S: for parameter counts far above Ns.
    linear=True follows the linear SSE (App. B): E_eff^lin in F, and ln Q of every trajectory
    integrated along with theta by the same scheme; lnq_out (a list) then receives ln Q at the
    measurement times as an array (n_meas, ntraj).
    """
    P, n = ans.P, ans.n
    n_ops = model.n_ops
    thetas, sigs, ms, qs, lqs = [], [], [], [], []
    w = tvmc.mc_weights(ns)
    for t in range(ntraj):
        tid = traj0 + t
        theta = np.zeros(P, complex) if theta0 is None else np.array(theta0, complex)
        sig = philox.initial_spins(seed, tid, ns, n)
        m_t, q_t, lq_t = [], [], []
        lnq = 0.0
        for i in range(n_steps):
            dW = philox.wiener_increments(seed, [tid], i, n_ops, dt)[0]
            g = [0.0, 0.0]

            def increment(th, stage):
                nonlocal sig
                sig, _ = tvmc.metropolis(ans, th, sig, seed, tid, 2 * i + stage, n_sweep)
                if stage == 0 and measure:
                    m, q = moments_from_samples(ans, th, sig, w)
                    m_t.append(m)
                    q_t.append(q)
                    lq_t.append(lnq)
                ev = tvmc.evaluate(model, ans, th, sig, w, dW, dt, with_S=not push, linear=linear)
                if linear:
                    g[stage] = tvmc.log_norm_increment(ev, w, dW, dt)
                if reg == "shift" and push:
                    return tvmc.solve_shift_push(ev["O"], tvmc.local_v(ev, dW, dt), w, eps)
                if reg == "shift":
                    return tvmc.solve_shift(ev["S"], ev["D"], eps)
                return tvmc.solve_snr(ev["S"], ev["D"], ev["O"], tvmc.local_v(ev, dW, dt), w)

            theta, _, _ = tvmc.sde_step(theta, increment, scheme)
            # the same scheme on ln Q: trapezoidal mean of the two increments, or the midpoint one
            lnq += 0.5 * (g[0] + g[1]) if scheme == "heun" else g[1]
        if measure:
            sig, _ = tvmc.metropolis(ans, theta, sig, seed, tid, 2 * n_steps, n_sweep)
            m, q = moments_from_samples(ans, theta, sig, w)
            m_t.append(m)
            q_t.append(q)
            lq_t.append(lnq)
        thetas.append(theta)
        sigs.append(sig)
        ms.append(m_t)
        qs.append(q_t)
        lqs.append(lq_t)
    if lnq_out is not None and measure:
        lnq_out.append(np.array(lqs).T)
    m = np.array(ms).transpose(1, 0, 2) if measure else None
    q = np.array(qs).transpose(1, 0, 2, 3) if measure else None
    return np.array(thetas), np.array(sigs), m, q


def run_enumeration(model, ans, ntraj, n_steps, dt, seed, scheme="heun", eps=1e-10, traj0=0, linear=False,
                    lnq_out=None):
    """Enumeration otVMC (exact expectations): per-step moments (n_steps+1, ntraj, ...).

    linear=True: the linear SSE with ln Q integrated alongside (see run_mc); lnq_out receives
    ln Q per step (n_steps+1, ntraj)."""
    from .tvmc import all_configs, exact_weights
    P, n = ans.P, ans.n
    sig = all_configs(n)
    ms, qs, thetas, lqs = [], [], [], []
    for t in range(ntraj):
        tid = traj0 + t
        theta = np.zeros(P, complex)
        m_t, q_t, lq_t = [], [], []
        lnq = 0.0
        for i in range(n_steps):
            w = exact_weights(ans, theta, sig)
            m, q = moments_from_samples(ans, theta, sig, w)
            m_t.append(m)
            q_t.append(q)
            lq_t.append(lnq)
            dW = philox.wiener_increments(seed, [tid], i, model.n_ops, dt)[0]
            g = [0.0, 0.0]

            def increment(th, stage):
                wt = exact_weights(ans, th, sig)
                ev = tvmc.evaluate(model, ans, th, sig, wt, dW, dt, linear=linear)
                if linear:
                    g[stage] = tvmc.log_norm_increment(ev, wt, dW, dt)
                return tvmc.solve_shift(ev["S"], ev["D"], eps)

            theta, _, _ = tvmc.sde_step(theta, increment, scheme)
            lnq += 0.5 * (g[0] + g[1]) if scheme == "heun" else g[1]
        w = exact_weights(ans, theta, sig)
        m, q = moments_from_samples(ans, theta, sig, w)
        m_t.append(m)
        q_t.append(q)
        lq_t.append(lnq)
        ms.append(m_t)
        qs.append(q_t)
        lqs.append(lq_t)
        thetas.append(theta)
    if lnq_out is not None:
        lnq_out.append(np.array(lqs).T)
    return np.array(thetas), np.array(ms).transpose(1, 0, 2), np.array(qs).transpose(1, 0, 2, 3)


def run_sse(model, ntraj, n_steps, dt, seed, scheme="heun", traj0=0, ito=False, linear=False, norm_out=None):
    """Exact-state trajectories of Eq. 4 (or Eq. 2 by Euler-Maruyama when ito=True); with
    linear=True of the linear SSE of App. B, whose moments are then the normalised ones and
    norm_out (a list) receives <psi|psi> per step (n_steps+1, ntraj)."""
    n = model.n
    H = dense_hamiltonian(model)
    Ls = dense_jump_ops(model)
    ms, qs, norms = [], [], []
    for t in range(ntraj):
        tid = traj0 + t
        psi = coherent_x_state(n)
        m_t, q_t, nr_t = [], [], []
        for i in range(n_steps):
            m, q = moments_from_state(psi, n)
            m_t.append(m)
            q_t.append(q)
            nr_t.append(np.vdot(psi, psi).real)
            dW = philox.wiener_increments(seed, [tid], i, model.n_ops, dt)[0]
            if linear:
                psi = sse.step_lin_ito_em(psi, H, Ls, dt, dW) if ito else sse.step_lin_strat(psi, H, Ls, dt, dW,
                                                                                               scheme)
            elif ito:
                psi = sse.step_ito_em(psi, H, Ls, dt, dW)
            else:
                psi = sse.step_strat(psi, H, Ls, dt, dW, scheme)
        m, q = moments_from_state(psi, n)
        m_t.append(m)
        q_t.append(q)
        nr_t.append(np.vdot(psi, psi).real)
        ms.append(m_t)
        qs.append(q_t)
        norms.append(nr_t)
    if norm_out is not None:
        norm_out.append(np.array(norms).T)
    return np.array(ms).transpose(1, 0, 2), np.array(qs).transpose(1, 0, 2, 3)
