"""Writes chain8_lindblad.txt: the exact magnetisation and spin moments of the 8-spin workload
(open chain, J_ij = 1/|i-j|^1.5, h = 1, decay kappa = 0.1 on every site, from the coherent state
along +x) from the oracle's RK4 integration of the Lindblad equation (Eq. 1), dt = 1e-3, at
t = 0, 0.1, ..., 1.0.  Columns: t, m_x, m_y, m_z, q_xx, q_yy, q_zz, q_xy, q_xz, q_yz.

    python tests/golden/make_chain8_lindblad.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lindblad  # noqa: E402
from oracle.model import Model, couplings, dense_hamiltonian, dense_jump_ops, coherent_x_state  # noqa: E402
from oracle.observables import moments_from_rho  # noqa: E402

OUT = os.path.join(HERE, "chain8_lindblad.txt")


def compute():
    n = 8
    model = Model(J=couplings((n,), 1.0, 1.5), h=1.0, kappa=np.full(n, 0.1), gamma=np.zeros(n))
    psi = coherent_x_state(n)
    dt, every = 1e-3, 100

    def obs(r):
        m, q = moments_from_rho(r, n)
        return np.concatenate([m, q[[0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]])
    _, recs = lindblad.evolve(np.outer(psi, psi.conj()), dense_hamiltonian(model), dense_jump_ops(model), 1.0, dt,
                              observe=obs, every=every)
    t = np.arange(len(recs)) * dt * every
    return np.column_stack([t, np.array(recs)])


if __name__ == "__main__":
    rows = compute()
    with open(OUT, "w") as f:
        f.write("# Exact Lindblad moments of the 8-spin workload (open chain, 1/r^1.5, h = 1, kappa = 0.1),\n")
        f.write("# written by make_chain8_lindblad.py from the oracle (RK4 of Eq. 1, dt = 1e-3).\n")
        f.write("# t m_x m_y m_z q_xx q_yy q_zz q_xy q_xz q_yz\n")
        for r in rows:
            f.write(" ".join(f"{v:.12e}" for v in r) + "\n")
    print(OUT)
