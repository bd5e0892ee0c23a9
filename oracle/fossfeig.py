"""Closed-form magnetisation and spin covariance of the 1D LITF model at h = 0 (App. D).

Test infrastructure (oracle side).  Periodic chain, quench from the coherent state along
+x, local decay at rate kappa, Gamma = kappa / 2.  The couplings enter through J_d, the
coupling at ring distance d (J_0 = 0, J_d = J_{N-d}); indices of J are taken mod N.

Sign reading: the formulas as printed agree with the exact Lindblad solution of
H = +sum_{i<j} J_{|i-j|} sz_i sz_j (signed couplings J_ij = +J_d in the library's
convention, with sy = [[0, -i], [i, 0]] in the (up, down) basis).  For the LITF sign of
Eq. 10, J_ij = -J_d, the y components (M_y, C_xy, C_yz) change sign and nothing else
does.  The oracle tests check this against the exact Lindblad solution at N <= 6.
"""
import numpy as np


def _phi(a, t, G):
    z = 2 * a * t + 1j * G * t
    return np.exp(-G * t) * (np.cos(z) + G / (2 * a + 1j * G) * np.sin(z))


def _psi(a, t, G):
    z = 2 * a * t + 1j * G * t
    return 2 * np.exp(-G * t) * (-G + 1j * a) / (2 * a + 1j * G) * np.sin(z)


def fossfeig(Jd, kappa, t):
    """M (3,), C (3, 3) at time t for ring couplings Jd[d], d = 0..N-1 (Jd[0] = 0).

    Phi(0) evaluates to 1 (0 * (1/0) form), handled by evaluating it as the limit.
    """
    Jd = np.asarray(Jd, dtype=np.float64)
    n = len(Jd)
    G = 0.5 * kappa

    def phi(a):
        a = np.asarray(a, dtype=np.float64)
        out = np.ones(a.shape, dtype=complex)
        nz = np.abs(2 * a + 1j * G) > 0
        out[nz] = _phi(a[nz], t, G)
        return out

    def psi(a):
        a = np.asarray(a, dtype=np.float64)
        out = np.zeros(a.shape, dtype=complex)
        nz = np.abs(2 * a + 1j * G) > 0
        out[nz] = _psi(a[nz], t, G)
        return out

    d = np.arange(n)
    Phi_mu = {mu: np.prod(phi(mu * Jd)) for mu in (1, -1)}
    Q_z = {}
    for mu in (1, -1):
        s = np.sum(psi(mu * Jd[1:]) / phi(mu * Jd[1:]))
        Q_z[mu] = np.exp(-G * t) / (2 * n) * Phi_mu[mu] * s
    Q = {}
    for mu in (1, -1):
        for nu in (1, -1):
            acc = 0.0 + 0.0j
            for D in range(1, n):
                num = np.prod(phi(mu * Jd + nu * Jd[(D - d) % n]))
                acc += num / (phi(mu * Jd[D]) * phi(nu * Jd[D]))
            Q[(mu, nu)] = np.exp(-2 * G * t) / (4 * n) * acc

    Mx = np.exp(-G * t) * Phi_mu[1].real
    My = np.exp(-G * t) * Phi_mu[1].imag
    Mz = np.exp(-2 * G * t) - 1.0
    C = np.zeros((3, 3))
    C[0, 0] = 1 / n + (2 * Q[(1, 1)] + Q[(-1, 1)] + Q[(1, -1)]).real - Mx ** 2
    C[1, 1] = 1 / n + (-2 * Q[(1, 1)] + Q[(-1, 1)] + Q[(1, -1)]).real - My ** 2
    C[0, 1] = C[1, 0] = 2 * Q[(1, 1)].imag - Mx * My
    C[0, 2] = C[2, 0] = (Q_z[1] + Q_z[-1]).real - Mx * Mz
    C[1, 2] = C[2, 1] = (Q_z[1] - Q_z[-1]).imag - My * Mz
    C[2, 2] = (1 / n) * (1 - Mz ** 2)
    return np.array([Mx, My, Mz]), C


def ring_couplings(n, J, alpha, kac=True):
    """J_d of App. D: (J/K(alpha)) |d|^-alpha with the nearest replica, J_0 = 0."""
    d = np.arange(n)
    r = np.minimum(d, n - d).astype(np.float64)
    Jd = np.zeros(n)
    Jd[1:] = J * r[1:] ** (-alpha)
    if kac:
        # Kac factor over all pairs of the ring (LITF paragraph, nearest replica)
        rr = np.minimum(np.abs(d[:, None] - d[None, :]), n - np.abs(d[:, None] - d[None, :]))
        iu = np.triu_indices(n, 1)
        K = np.sum(rr[iu].astype(float) ** (-alpha)) / (n - 1)
        Jd /= K
    return Jd
