"""Variational wavefunctions of the otVMC method: long-range Jastrow (Eq. 12), its partially
inhomogeneous variants LJPHd / LJH (paragraph after Eq. 12) and RBM (Eq. 11).

Test infrastructure (oracle side).  sig is an integer array (Ns, N) of sigma_j in {-1, +1}
(eigenvalues of sz_j, LITF paragraph); theta is a complex vector (P,).

Parameter layouts (interface with the CUDA library, shared as a convention only):
* Jastrow, P = N(N+1)/2: theta = [a_0 .. a_{N-1}, eta_jk for j < k in row-major order
  (0,1), (0,2), .., (0,N-1), (1,2), .., (N-2,N-1)].
  log psi = sum_i a_i sigma_i + sum_{j<k} eta_jk sigma_j sigma_k       (Eq. 12)
* LJPHd / LJH (tied Jastrow): theta = [a_0 .. a_{N-1}, one eta per group of pairs], the
  groups from lj_groups: the pairs at distance <= d one by one in row-major order, then the
  pairs of each larger distance together, in increasing distance.  P = N + number of groups.
* RBM with M hidden units, P = N + M + N M: theta = [a (N), b (M), W (N x M row-major)].
  log psi = sum_i a_i sigma_i + sum_m log(2 cosh gamma_m),
  gamma_m = b_m + sum_i W_im sigma_i                                    (Eq. 11)

Local operators O_k(x) = d log psi(x) / d theta_k (definitions after Eq. 8).
Flip ratios r_j(x) = psi(x with sigma_j -> -sigma_j) / psi(x) are returned as logs.
"""
import numpy as np


def log2cosh(z):
    """log(2 cosh z) = s z + log(1 + exp(-2 s z)), s = sign(Re z): no overflow."""
    z = np.asarray(z, dtype=complex)
    s = np.where(z.real >= 0, 1.0, -1.0)
    return s * z + np.log1p(np.exp(-2.0 * s * z))


class Jastrow:
    kind = "jastrow"

    def __init__(self, n):
        self.n = n
        self.P = n * (n + 1) // 2
        self.pairs = np.array([(j, k) for j in range(n) for k in range(j + 1, n)], dtype=np.int64)

    def split(self, theta):
        n = self.n
        a = theta[:n]
        eta = np.zeros((n, n), dtype=complex)
        eta[self.pairs[:, 0], self.pairs[:, 1]] = theta[n:]
        eta = eta + eta.T
        return a, eta

    def logpsi(self, theta, sig):
        a, eta = self.split(theta)
        s = sig.astype(np.float64)
        return s @ a + 0.5 * np.einsum("xj,jk,xk->x", s, eta, s)

    def O(self, theta, sig):
        s = sig.astype(np.float64)
        return np.concatenate([s, s[:, self.pairs[:, 0]] * s[:, self.pairs[:, 1]]], axis=1).astype(complex)

    def log_flip_ratios(self, theta, sig):
        """log r_j = -2 sigma_j (a_j + sum_{k != j} eta_jk sigma_k)."""
        a, eta = self.split(theta)
        s = sig.astype(np.float64)
        field = a[None, :] + s @ eta.T        # eta has zero diagonal
        return -2.0 * s * field

    def log_pair_flip_ratios(self, theta, sig):
        """log psi(x^(jk)) / psi(x) for all j != k: log r_j + log r_k + 4 sigma_j sigma_k eta_jk."""
        a, eta = self.split(theta)
        s = sig.astype(np.float64)
        lr = self.log_flip_ratios(theta, sig)
        return lr[:, :, None] + lr[:, None, :] + 4.0 * s[:, :, None] * s[:, None, :] * eta[None]


def lj_groups(n, d, pbc=False):
    """Parameter groups of the partially inhomogeneous long-range Jastrow LJPHd (Eq. 12 and the
    paragraph after it): eta_jk is free for every pair at distance D <= d and shared by all
    pairs at the same distance D > d.  D = |j - k| for an open chain, or the nearest-image
    distance min(|j - k|, N - |j - k|) for a periodic one (pbc).  d = 0 is the homogeneous LJH,
    d >= the largest distance the fully inhomogeneous LJNH (the full Jastrow).

    Returns a list of groups, each a list of pairs (j, k) with j < k: first one group per free
    pair in row-major order, then one group per shared distance in increasing order.
    """
    def dist(j, k):
        D = k - j
        return min(D, n - D) if pbc else D
    pairs = [(j, k) for j in range(n) for k in range(j + 1, n)]
    groups = [[p] for p in pairs if dist(*p) <= d]
    for D in sorted({dist(*p) for p in pairs if dist(*p) > d}):
        groups.append([p for p in pairs if dist(*p) == D])
    return groups


class TiedJastrow:
    """Long-range Jastrow (Eq. 12) whose two-body parameters are shared within groups of pairs.

    theta = [a_0 .. a_{N-1}, eta_g for each group g]; log psi = sum_i a_i sigma_i +
    sum_g eta_g sum_{(j,k) in g} sigma_j sigma_k, so O_{eta_g} = sum_{(j,k) in g} sigma_j sigma_k
    and the flip ratios are those of the full Jastrow with eta_jk = eta_g(j,k).
    """
    kind = "jastrow"

    def __init__(self, n, groups):
        self.n = n
        self.groups = [list(g) for g in groups]
        self.P = n + len(self.groups)
        self.gidx = np.full((n, n), -1, dtype=np.int64)
        for g, grp in enumerate(self.groups):
            for j, k in grp:
                self.gidx[j, k] = self.gidx[k, j] = g

    def split(self, theta):
        """(a, eta) with eta the full symmetric N x N matrix of the expanded pair parameters."""
        n = self.n
        a = theta[:n]
        eta = np.zeros((n, n), dtype=complex)
        off = self.gidx >= 0
        eta[off] = theta[n + self.gidx[off]]
        return a, eta

    def logpsi(self, theta, sig):
        a, eta = self.split(theta)
        s = sig.astype(np.float64)
        return s @ a + 0.5 * np.einsum("xj,jk,xk->x", s, eta, s)

    def O(self, theta, sig):
        s = sig.astype(np.float64)
        cols = [s[:, [j for j, _ in g]] * s[:, [k for _, k in g]] for g in self.groups]
        two = np.stack([c.sum(axis=1) for c in cols], axis=1) if cols else np.zeros((s.shape[0], 0))
        return np.concatenate([s, two], axis=1).astype(complex)

    def log_flip_ratios(self, theta, sig):
        a, eta = self.split(theta)
        s = sig.astype(np.float64)
        return -2.0 * s * (a[None, :] + s @ eta.T)

    def log_pair_flip_ratios(self, theta, sig):
        a, eta = self.split(theta)
        s = sig.astype(np.float64)
        lr = self.log_flip_ratios(theta, sig)
        return lr[:, :, None] + lr[:, None, :] + 4.0 * s[:, :, None] * s[:, None, :] * eta[None]


def lj_ansatz(n, d, pbc=False):
    """LJPHd on N sites (LJH for d = 0)."""
    return TiedJastrow(n, lj_groups(n, d, pbc))


class RBM:
    kind = "rbm"

    def __init__(self, n, m):
        self.n, self.m = n, m
        self.P = n + m + n * m

    def split(self, theta):
        n, m = self.n, self.m
        return theta[:n], theta[n:n + m], theta[n + m:].reshape(n, m)

    def angles(self, theta, sig):
        a, b, W = self.split(theta)
        return b[None, :] + sig.astype(np.float64) @ W

    def logpsi(self, theta, sig):
        a, b, W = self.split(theta)
        return sig.astype(np.float64) @ a + log2cosh(self.angles(theta, sig)).sum(axis=1)

    def O(self, theta, sig):
        s = sig.astype(np.float64)
        t = np.tanh(self.angles(theta, sig))
        ns = s.shape[0]
        return np.concatenate([s.astype(complex), t, (s[:, :, None] * t[:, None, :]).reshape(ns, -1)], axis=1)

    def log_flip_ratios(self, theta, sig):
        """log r_j = -2 a_j sigma_j + sum_m [lc(gamma_m - 2 W_jm sigma_j) - lc(gamma_m)]."""
        a, b, W = self.split(theta)
        s = sig.astype(np.float64)
        g = self.angles(theta, sig)
        lc0 = log2cosh(g)
        g1 = g[:, None, :] - 2.0 * s[:, :, None] * W[None, :, :]
        return -2.0 * a[None, :] * s + (log2cosh(g1) - lc0[:, None, :]).sum(axis=2)

    def log_pair_flip_ratios(self, theta, sig):
        a, b, W = self.split(theta)
        s = sig.astype(np.float64)
        g = self.angles(theta, sig)
        lc0 = log2cosh(g).sum(axis=1)
        dW = 2.0 * s[:, :, None] * W[None, :, :]             # (Ns, N, M)
        g2 = g[:, None, None, :] - dW[:, :, None, :] - dW[:, None, :, :]
        da = -2.0 * a[None, :] * s
        return da[:, :, None] + da[:, None, :] + log2cosh(g2).sum(axis=3) - lc0[:, None, None]


def make_ansatz(kind, n, m=0, d=0, pbc=False):
    if kind == "lj":
        return lj_ansatz(n, d, pbc)
    return Jastrow(n) if kind == "jastrow" else RBM(n, m)
