"""Magnetisation, spin covariance and Wineland squeezing (LITF paragraph, Eq. 3).

Test infrastructure (oracle side).

Per trajectory, from configurations with weights w (MC 1/Ns or exact |psi|^2/Z):
  m_a   = (1/N) sum_j <s^a_j>                         a in {x, y, z}
  q_ab  = (1/N^2) sum_{j,k} <(s^a_j s^b_k + s^b_k s^a_j)/2>
with the local estimators (sigma_j = +-1, r_j flip ratio, r_jk two-flip ratio, j != k)
  s^x_j -> r_j,  s^y_j -> -i sigma_j r_j,  s^z_j -> sigma_j,
  s^x_j s^x_k -> r_jk,  s^y_j s^y_k -> -sigma_j sigma_k r_jk,  s^x_j s^y_k -> -i sigma_k r_jk,
  s^x_j s^z_k -> sigma_k r_j,  s^y_j s^z_k -> -i sigma_j sigma_k r_j,  s^z_j s^z_k -> sigma_j sigma_k,
and the same-site terms s^a s^b + s^b s^a = 2 delta_ab.  Real parts are taken (the
exact values are real).  The ensemble (Eq. 3) averages m and q over trajectories; then
M = <m>, C = <q> - M M^T (normalised spin covariance), and
xi^2 = N min_perp Var(M_perp) / |M|^2 over the plane perpendicular to M (Wineland).
"""
import numpy as np


def moments_from_samples(ans, theta, sig, w):
    s = sig.astype(np.float64)
    n = s.shape[1]
    r = np.exp(ans.log_flip_ratios(theta, sig))
    r2 = np.exp(ans.log_pair_flip_ratios(theta, sig))
    off = ~np.eye(n, dtype=bool)
    E = lambda X: np.tensordot(w, X, axes=(0, 0))
    m = np.array([E(r).sum().real, E(-1j * s * r).sum().real, E(s).sum().real]) / n
    ss = s[:, :, None] * s[:, None, :]
    pair = {
        (0, 0): r2,
        (1, 1): -ss * r2,
        (0, 1): -1j * s[:, None, :] * r2,
        (0, 2): s[:, None, :] * r[:, :, None],
        (1, 2): -1j * ss * r[:, :, None],
        (2, 2): ss.astype(complex),
    }
    q = np.zeros((3, 3))
    for (a, b), X in pair.items():
        val = (E(X)[off]).sum().real
        q[a, b] = q[b, a] = val
    q += n * np.eye(3)
    return m, q / n ** 2


def moments_from_state(psi, n):
    """Exact m, q of a state vector (dense Pauli operators)."""
    from .model import pauli_ops
    ops = [pauli_ops(n, j)[:3] for j in range(n)]
    M = [sum(o[a] for o in ops) / n for a in range(3)]
    nrm = np.vdot(psi, psi).real
    m = np.array([np.vdot(psi, A @ psi).real / nrm for A in M])
    q = np.array([[0.5 * np.vdot(psi, (A @ B + B @ A) @ psi).real / nrm for B in M] for A in M])
    return m, q


def moments_from_rho(rho, n):
    from .model import pauli_ops
    ops = [pauli_ops(n, j)[:3] for j in range(n)]
    M = [sum(o[a] for o in ops) / n for a in range(3)]
    m = np.array([np.trace(A @ rho).real for A in M])
    q = np.array([[0.5 * np.trace((A @ B + B @ A) @ rho).real for B in M] for A in M])
    return m, q


def ensemble(m_traj, q_traj):
    """Eq. 3 averages: M, C and their standard errors over trajectories."""
    m_traj = np.asarray(m_traj)
    q_traj = np.asarray(q_traj)
    nt = m_traj.shape[0]
    M = m_traj.mean(axis=0)
    Q = q_traj.mean(axis=0)
    C = Q - np.outer(M, M)
    dM = m_traj.std(axis=0, ddof=1) / np.sqrt(nt) if nt > 1 else np.zeros(3)
    return M, C, dM


def ensemble_weighted(m_traj, q_traj, Q):
    """Eq. 3 for the linear SSE (App. B): the normalised moments of each trajectory weighted by
    its norm Q_j, M = (1/N_T) sum_j Q_j m_j, <q> likewise, C = <q> - M M^T; standard errors of M
    from the weighted samples Q_j m_j."""
    m_traj = np.asarray(m_traj)
    q_traj = np.asarray(q_traj)
    Q = np.asarray(Q, dtype=np.float64)
    nt = m_traj.shape[0]
    mw = Q[:, None] * m_traj
    M = mw.mean(axis=0)
    C = (Q[:, None, None] * q_traj).mean(axis=0) - np.outer(M, M)
    dM = mw.std(axis=0, ddof=1) / np.sqrt(nt) if nt > 1 else np.zeros(3)
    return M, C, dM


def squeezing(M, C, n):
    """xi^2 = N lambda_min(C restricted to the plane perpendicular to M) / |M|^2."""
    M = np.asarray(M, dtype=np.float64)
    nrm = np.linalg.norm(M)
    u = M / nrm
    # orthonormal basis of the perpendicular plane
    trial = np.eye(3)[np.argmin(np.abs(u))]
    e1 = trial - u * (trial @ u)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u, e1)
    P = np.stack([e1, e2])
    Cp = P @ C @ P.T
    return n * np.linalg.eigvalsh(Cp)[0] / nrm ** 2
