"""Shared set-up of the GPU parity tests: the same model and inputs on both sides.

Inputs come from the seeded generators in `synth`; expected values come from `oracle`.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle.model import Model as OModel, couplings  # noqa: E402
from oracle.ansatz import Jastrow  # noqa: E402


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23928_gb300 import build
    build.build()


class Case:
    """A model/ansatz pair on the library and on the oracle, plus tensors helpers."""

    def __init__(self, extent, alpha=1.5, h=1.0, kappa=0.1, gamma=0.0, J=1.0, pbc=False):
        import paper_2506_23928_gb300 as pkg
        self.J = couplings(extent, J, alpha, pbc=pbc)
        self.n = self.J.shape[0]
        self.kappa = np.broadcast_to(np.asarray(kappa, float), (self.n,)).copy()
        self.gamma = np.broadcast_to(np.asarray(gamma, float), (self.n,)).copy()
        self.omodel = OModel(J=self.J, h=h, kappa=self.kappa, gamma=self.gamma)
        self.oans = Jastrow(self.n)
        self.model = pkg.Model(self.J, h, self.kappa, self.gamma)
        self.ans = pkg.Ansatz(self.model)
        self.P = self.ans.P
        self.nops = self.model.nops
        self.W = (self.n + 63) // 64
        assert self.P == self.oans.P and self.nops == self.omodel.n_ops

    def theta(self, seed, ntraj, scale=0.05):
        th = synth.random_theta(seed, ntraj, self.P, scale)
        return th, to_dev_complex(th)

    def spins(self, seed, ntraj, ns):
        sig = synth.random_spins(seed, ntraj, ns, self.n)
        return sig, torch.from_numpy(synth.pack_spins(sig).view(np.int64)).cuda()

    def work(self, ntraj, ns, precision):
        from paper_2506_23928_gb300 import abi
        nb = abi.otvmc_workspace_bytes(self.ans.handle, ntraj, ns, precision)
        assert nb > 0
        return torch.zeros(nb, dtype=torch.uint8, device="cuda"), nb


def to_dev_complex(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return torch.from_numpy(a.view(np.float64).copy()).cuda()


def from_dev_complex(t):
    return t.cpu().numpy().view(np.complex128)


def unpack(t, n):
    return synth.unpack_spins(t.cpu().numpy().view(np.uint64), n)


def rel_err(got, want):
    got, want = np.asarray(got), np.asarray(want)
    den = np.abs(want).max()
    return np.abs(got - want).max() / (den if den > 0 else 1.0)
