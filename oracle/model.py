"""Lindblad model of the otVMC method: Hamiltonian, jump operators, dense operators.

Test infrastructure (oracle side): plain numpy FP64, no blocking or fusion.

* Hamiltonian of the long-range Ising model in a transverse field (Eq. 10).  The library
  takes explicit signed couplings: H = sum_{i<j} J_ij sz_i sz_j + h sum_i sx_i.  The
  paper's form, -(J/K(alpha)) sum sz sz / |i-j|^alpha - h sum sx, is the special case
  J_ij = -J / (K r_ij^alpha) with h -> -h.  K(alpha) = sum_{i<j} r_ij^-alpha / (N - 1)
  is the Kac factor of the same paragraph.
* Jump operators: local decay L_i = sqrt(kappa_i) s^-_i (the LITF paragraph) and local
  dephasing L_i = sqrt(gamma_i) sz_i.  Operators with zero rate are left out.  Order:
  all decay operators in site order, then all dephasing operators in site order.
* Basis: configuration index x in [0, 2^N); bit j of x set <=> sigma_j = +1 (spin up,
  eigenvalue +1 of sz_j).  s^- maps up to down.
"""
from dataclasses import dataclass, field
import numpy as np


def lattice_coords(extent):
    """Integer site coordinates of an open 1D chain or 2D square lattice (row-major)."""
    extent = list(extent)
    if len(extent) == 1:
        return np.arange(extent[0], dtype=np.float64)[:, None]
    lx, ly = extent
    ii, jj = np.meshgrid(np.arange(lx), np.arange(ly), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.float64)


def distances(extent, pbc):
    """Pairwise distances; with pbc the nearest periodic image along each axis."""
    extent = np.asarray(list(extent), dtype=np.float64)
    x = lattice_coords(extent.astype(int))
    d = np.abs(x[:, None, :] - x[None, :, :])
    if pbc:
        d = np.minimum(d, extent[None, None, :] - d)
    return np.sqrt((d ** 2).sum(axis=-1))


def kac_factor(r, alpha):
    """K(alpha) = sum_{i<j} r_ij^-alpha / (N - 1)  (LITF paragraph)."""
    n = r.shape[0]
    iu = np.triu_indices(n, 1)
    return np.sum(r[iu] ** (-alpha)) / (n - 1)


def couplings(extent, J, alpha, kac=False, pbc=False):
    """J_ij = J / r_ij^alpha (divided by K(alpha) when kac), zero diagonal."""
    r = distances(extent, pbc)
    n = r.shape[0]
    out = np.zeros((n, n))
    off = ~np.eye(n, dtype=bool)
    out[off] = J * r[off] ** (-alpha)
    if kac:
        out /= kac_factor(r, alpha)
    return out


@dataclass
class Model:
    """H = sum_{i<j} J_ij sz_i sz_j + h sum_i sx_i, jump operators from per-site rates."""
    J: np.ndarray
    h: float
    kappa: np.ndarray
    gamma: np.ndarray
    n: int = field(init=False)

    def __post_init__(self):
        self.J = np.asarray(self.J, dtype=np.float64)
        self.n = self.J.shape[0]
        self.kappa = np.broadcast_to(np.asarray(self.kappa, dtype=np.float64), (self.n,)).copy()
        self.gamma = np.broadcast_to(np.asarray(self.gamma, dtype=np.float64), (self.n,)).copy()
        assert np.allclose(self.J, self.J.T) and np.all(np.diag(self.J) == 0)

    def jump_ops(self):
        """List of (kind, site, rate) with kind 'decay' or 'dephase', zero rates dropped."""
        ops = [("decay", j, self.kappa[j]) for j in range(self.n) if self.kappa[j] > 0]
        ops += [("dephase", j, self.gamma[j]) for j in range(self.n) if self.gamma[j] > 0]
        return ops

    @property
    def n_ops(self):
        return len(self.jump_ops())


# ---------------------------------------------------------------- dense operators (small N)

def spins_of_index(n):
    """sigma[x, j] in {-1, +1} for every basis index x (bit j set <=> +1)."""
    x = np.arange(2 ** n)[:, None]
    return np.where((x >> np.arange(n)[None, :]) & 1, 1, -1).astype(np.int64)


def pauli_ops(n, j):
    """Dense sx_j, sy_j, sz_j, s^-_j on the 2^N basis (as (d, d) complex arrays)."""
    d = 2 ** n
    x = np.arange(d)
    up = ((x >> j) & 1) == 1
    y = x ^ (1 << j)
    sx = np.zeros((d, d), complex)
    sx[x, y] = 1.0
    sy = np.zeros((d, d), complex)
    # <x| sy |y>: sy|up> = i|down>, sy|down> = -i|up>
    sy[y, x] = np.where(up, 1j, -1j)
    sz = np.diag(np.where(up, 1.0, -1.0)).astype(complex)
    sm = np.zeros((d, d), complex)
    sm[y[up], x[up]] = 1.0          # s^- |up> = |down>
    return sx, sy, sz, sm


def dense_hamiltonian(model):
    n = model.n
    sig = spins_of_index(n).astype(np.float64)
    diag = 0.5 * np.einsum("xi,ij,xj->x", sig, model.J, sig)
    H = np.diag(diag).astype(complex)
    for j in range(n):
        H += model.h * pauli_ops(n, j)[0]
    return H


def dense_jump_ops(model):
    out = []
    for kind, j, rate in model.jump_ops():
        sx, sy, sz, sm = pauli_ops(model.n, j)
        out.append(np.sqrt(rate) * (sm if kind == "decay" else sz))
    return out


def coherent_x_state(n):
    """|+x>^N, the initial state of every quench (LITF paragraph)."""
    d = 2 ** n
    return np.full(d, d ** -0.5, dtype=complex)
