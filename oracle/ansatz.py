"""Variational wavefunctions of the otVMC method: long-range Jastrow (Eq. 12) and RBM (Eq. 11).

Test infrastructure (oracle side).  sig is an integer array (Ns, N) of sigma_j in {-1, +1}
(eigenvalues of sz_j, LITF paragraph); theta is a complex vector (P,).

Parameter layouts (interface with the CUDA library, shared as a convention only):
* Jastrow, P = N(N+1)/2: theta = [a_0 .. a_{N-1}, eta_jk for j < k in row-major order
  (0,1), (0,2), .., (0,N-1), (1,2), .., (N-2,N-1)].
  log psi = sum_i a_i sigma_i + sum_{j<k} eta_jk sigma_j sigma_k       (Eq. 12)
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


def make_ansatz(kind, n, m=0):
    return Jastrow(n) if kind == "jastrow" else RBM(n, m)
