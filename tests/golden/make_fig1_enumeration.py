"""Writes fig1_enumeration.txt: the paper's N = 10 setup (Fig. 1: periodic ring, alpha = 1 with the
Kac factor, the LITF sign J_ij = -J_d, h = 0, decay kappa = 0.5 on every site, from the coherent
state along +x) run by the oracle's enumeration otVMC (exact expectations over all 2^10
configurations, no sampling) with the full Jastrow ansatz, shift 1e-3, midpoint, dt = 0.005, on
the Wiener increments of seed 3 for trajectories 0..399.  Rows t = 0, 0.1, .., 0.8; columns t,
M_x, M_y, M_z, xi^2 of the ensemble (Eq. 3, Wineland xi^2).

    python tests/golden/make_fig1_enumeration.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
OUT = os.path.join(HERE, "fig1_enumeration.txt")
N, KAPPA, DT, TMAX, EPS, SEED, NTRAJ = 10, 0.5, 0.005, 0.8, 1e-3, 3, 400


def _model():
    from oracle import fossfeig
    from oracle.model import Model
    Jd = fossfeig.ring_couplings(N, 1.0, 1.0, kac=True)
    Jij = np.array([[0.0 if i == j else -Jd[(i - j) % N] for j in range(N)] for i in range(N)])
    return Model(J=Jij, h=0.0, kappa=np.full(N, KAPPA), gamma=np.zeros(N))


def _chunk(args):
    t0, cnt = args
    from oracle import trajectories as tr
    from oracle.ansatz import Jastrow
    steps = int(round(TMAX / DT))
    _, M, Q = tr.run_enumeration(_model(), Jastrow(N), cnt, steps, DT, SEED, "midpoint", eps=EPS, traj0=t0)
    return M, Q


def compute(procs=8):
    from oracle.observables import ensemble, squeezing
    chunks = [(k, min(10, NTRAJ - k)) for k in range(0, NTRAJ, 10)]
    with mp.get_context("spawn").Pool(procs) as p:
        res = p.map(_chunk, chunks)
    M = np.concatenate([r[0] for r in res], axis=1)
    Q = np.concatenate([r[1] for r in res], axis=1)
    every = int(round(0.1 / DT))
    rows = []
    for i in range(0, M.shape[0], every):
        Me, C, _ = ensemble(M[i], Q[i])
        rows.append([i * DT, *Me, squeezing(Me, C, N) if i > 0 else 1.0])
    return np.array(rows)


if __name__ == "__main__":
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    rows = compute()
    with open(OUT, "w") as f:
        f.write("# Enumeration otVMC (exact expectations) of the N = 10 setup of Fig. 1, full Jastrow, shift 1e-3,\n")
        f.write("# midpoint, dt = 0.005, Wiener increments of seed 3, trajectories 0..399; written by\n")
        f.write("# make_fig1_enumeration.py from the oracle.  t M_x M_y M_z xi2\n")
        for r in rows:
            f.write(" ".join(f"{v:.12e}" for v in r) + "\n")
    print(OUT)
