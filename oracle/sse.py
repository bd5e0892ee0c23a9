"""Exact-state quantum trajectories of the nonlinear and the linear stochastic Schroedinger
equation.

Test infrastructure (oracle side).  State vectors psi in C^(2^N), small N only.

* Ito form (Eq. 2), integrated by Euler-Maruyama:
    dpsi = {[-iH - 1/2 sum_n (L^+L - <L+L^+> L + 1/4 <L+L^+>^2)] dt
            + sum_n (L - 1/2 <L+L^+>) dW_n} psi.
* Stratonovich form (Eq. 4 with the effective Hamiltonian Eq. 5), integrated by the
  predictor-corrector schemes of App. C (trapezoidal / Heun and midpoint), all with the
  same Delta W for predictor and corrector:
    dpsi = [-i H_eff dt + sum_n (L - 1/2 <L+L^+>) o dW_n] psi,
    H_eff = H - i/2 sum_n (L^+L - 2<L+L^+> L + L^2 + <L+L^+>^2 - 1/2 <L^2 + 2 L^+L + L^+2>).
Expectations <.> are taken in the normalised state (Eq. 2 preserves the norm; the
discrete schemes only to O(dt)).  Trajectory averages follow Eq. 3.
* Linear SSE (App. B): Ito form dpsi = [(-iH - 1/2 sum L^+L) dt + sum L dW] psi, Stratonovich
  form dpsi = [-i H_lin dt + sum L o dW] psi with H_lin = H - i/2 sum (L^+L + L^2).  The state
  is not normalised; Eq. 3 holds with unnormalised expectations <psi|A|psi>.
"""
import numpy as np


def expect(psi, A):
    return np.vdot(psi, A @ psi) / np.vdot(psi, psi)


def _lpl(psi, L):
    return (expect(psi, L + L.conj().T)).real


def ito_drift_diffusion(psi, H, Ls):
    drift = -1j * (H @ psi)
    diff = []
    for L in Ls:
        m = _lpl(psi, L)
        drift += -0.5 * (L.conj().T @ (L @ psi) - m * (L @ psi) + 0.25 * m * m * psi)
        diff.append(L @ psi - 0.5 * m * psi)
    return drift, diff


def strat_drift_diffusion(psi, H, Ls):
    """A(psi) = -i H_eff psi and B_n(psi) = (L_n - <L_n+L_n^+>/2) psi (Eqs. 4-5)."""
    Heff_psi = H @ psi
    diff = []
    for L in Ls:
        Ld = L.conj().T
        m = _lpl(psi, L)
        Lpsi = L @ psi
        LdLpsi = Ld @ Lpsi
        L2psi = L @ Lpsi
        c = m * m - 0.5 * expect(psi, L @ L + 2 * Ld @ L + Ld @ Ld)
        Heff_psi = Heff_psi - 0.5j * (LdLpsi - 2 * m * Lpsi + L2psi + c * psi)
        diff.append(Lpsi - 0.5 * m * psi)
    return -1j * Heff_psi, diff


def step_ito_em(psi, H, Ls, dt, dW):
    a, b = ito_drift_diffusion(psi, H, Ls)
    return psi + a * dt + sum(bn * w for bn, w in zip(b, dW))


def step_strat(psi, H, Ls, dt, dW, scheme="heun"):
    """One step of App. C on the state vector (predictor X-bar, then corrector)."""
    a0, b0 = strat_drift_diffusion(psi, H, Ls)
    incr0 = a0 * dt + sum(bn * w for bn, w in zip(b0, dW))
    pred = psi + incr0
    if scheme == "heun":
        a1, b1 = strat_drift_diffusion(pred, H, Ls)
        incr1 = a1 * dt + sum(bn * w for bn, w in zip(b1, dW))
        return psi + 0.5 * (incr0 + incr1)
    if scheme == "midpoint":
        a1, b1 = strat_drift_diffusion(0.5 * (psi + pred), H, Ls)
        return psi + a1 * dt + sum(bn * w for bn, w in zip(b1, dW))
    raise ValueError(scheme)


def lin_strat_drift_diffusion(psi, H, Ls):
    """A(psi) = -i H_lin psi, B_n(psi) = L_n psi (linear SSE, App. B)."""
    Hpsi = H @ psi
    diff = []
    for L in Ls:
        Lpsi = L @ psi
        Hpsi = Hpsi - 0.5j * (L.conj().T @ Lpsi + L @ Lpsi)
        diff.append(Lpsi)
    return -1j * Hpsi, diff


def step_lin_ito_em(psi, H, Ls, dt, dW):
    drift = -1j * (H @ psi) - 0.5 * sum(L.conj().T @ (L @ psi) for L in Ls)
    return psi + drift * dt + sum((L @ psi) * w for L, w in zip(Ls, dW))


def step_lin_strat(psi, H, Ls, dt, dW, scheme="heun"):
    """One predictor-corrector step (App. C) of the linear Stratonovich SSE."""
    a0, b0 = lin_strat_drift_diffusion(psi, H, Ls)
    incr0 = a0 * dt + sum(bn * w for bn, w in zip(b0, dW))
    pred = psi + incr0
    if scheme == "heun":
        a1, b1 = lin_strat_drift_diffusion(pred, H, Ls)
        return psi + 0.5 * (incr0 + a1 * dt + sum(bn * w for bn, w in zip(b1, dW)))
    if scheme == "midpoint":
        a1, b1 = lin_strat_drift_diffusion(0.5 * (psi + pred), H, Ls)
        return psi + a1 * dt + sum(bn * w for bn, w in zip(b1, dW))
    raise ValueError(scheme)
