"""Exact density-matrix dynamics (Eq. 1) for small N: the physical truth otVMC approximates.

Test infrastructure (oracle side).  d rho/dt = -i[H, rho] + sum_n (L rho L^+ - 1/2 {L^+ L, rho})
(Eq. 1, hbar = 1) integrated by the classical fourth-order Runge-Kutta method with a
fixed step; observables are Tr(A rho) (the double-bracket expectation under Eq. 1).
The dense Liouvillian (for scipy's matrix exponential at N <= 3) is built from the same
equation written as a 4^N x 4^N matrix acting on row-major vec(rho).
"""
import numpy as np


def lindblad_rhs(rho, H, Ls):
    out = -1j * (H @ rho - rho @ H)
    for L in Ls:
        Ld = L.conj().T
        LdL = Ld @ L
        out += L @ rho @ Ld - 0.5 * (LdL @ rho + rho @ LdL)
    return out


def evolve(rho0, H, Ls, t_final, dt, observe=None, every=1):
    """RK4 from rho0 to t_final; observe(rho) recorded at t = 0, every*dt, ..."""
    n_steps = int(round(t_final / dt))
    rho = rho0.copy()
    recs = [observe(rho)] if observe else []
    for s in range(n_steps):
        k1 = lindblad_rhs(rho, H, Ls)
        k2 = lindblad_rhs(rho + 0.5 * dt * k1, H, Ls)
        k3 = lindblad_rhs(rho + 0.5 * dt * k2, H, Ls)
        k4 = lindblad_rhs(rho + dt * k3, H, Ls)
        rho = rho + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        if observe and (s + 1) % every == 0:
            recs.append(observe(rho))
    return rho, recs


def liouvillian(H, Ls):
    """Matrix of Eq. 1 acting on row-major vec(rho): vec(A rho B) = (A kron B^T) vec(rho)."""
    d = H.shape[0]
    I = np.eye(d)
    Lv = -1j * (np.kron(H, I) - np.kron(I, H.T))
    for L in Ls:
        Ld = L.conj().T
        LdL = Ld @ L
        Lv += np.kron(L, L.conj()) - 0.5 * (np.kron(LdL, I) + np.kron(I, LdL.T))
    return Lv
