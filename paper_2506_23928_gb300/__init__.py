"""GB300 (sm_103a) implementation of the otVMC hot path (arXiv:2506.23928) behind a C ABI.

The compute path is libotvmc.so (CUDA C++, include/otvmc.h).  This package holds its
ctypes binding (`abi`, the C entry points under the same names), its build script
(`build`), and two small handle wrappers used by the tests and the benchmark.
"""
import ctypes

import numpy as np

from . import abi
from .abi import check


class Model:
    """otvmc_model handle: H = sum_{i<j} J_ij sz_i sz_j + h sum_i sx_i, decay and dephasing."""

    def __init__(self, J, h, kappa=None, gamma=None):
        J = np.ascontiguousarray(J, dtype=np.float64)
        n = J.shape[0]
        self._keep = [J]
        kp = gp = None
        if kappa is not None:
            kp = np.ascontiguousarray(np.broadcast_to(np.asarray(kappa, dtype=np.float64), (n,)))
            self._keep.append(kp)
        if gamma is not None:
            gp = np.ascontiguousarray(np.broadcast_to(np.asarray(gamma, dtype=np.float64), (n,)))
            self._keep.append(gp)
        desc = abi.ModelDesc(n, J.ctypes.data, float(h), kp.ctypes.data if kp is not None else None,
                             gp.ctypes.data if gp is not None else None)
        out = ctypes.c_void_p()
        check(abi.otvmc_model_create(desc, out))
        self.handle = out.value
        self.n = n
        self.nops = abi.otvmc_model_nops(self.handle)

    def __del__(self):
        if getattr(self, "handle", None):
            abi.otvmc_model_destroy(self.handle)
            self.handle = None


class Ansatz:
    """otvmc_ansatz handle: Jastrow (Eq. 12), RBM with n_hidden hidden units (Eq. 11), or the tied
    Jastrow LJPHd (kind OTVMC_LJ, tie distance d, nearest-image distances when pbc)."""

    def __init__(self, model, kind=abi.OTVMC_JASTROW, n_hidden=0, d=0, pbc=False):
        out = ctypes.c_void_p()
        if kind == abi.OTVMC_LJ:
            check(abi.otvmc_ansatz_create_lj(model.handle, d, int(pbc), out))
        else:
            check(abi.otvmc_ansatz_create(model.handle, kind, n_hidden, out))
        self.handle = out.value
        self.model = model
        self.n = model.n
        self.P = abi.otvmc_ansatz_nparams(self.handle)

    def __del__(self):
        if getattr(self, "handle", None):
            abi.otvmc_ansatz_destroy(self.handle)
            self.handle = None


def lattice_couplings(extent, J, alpha, kac=False, pbc=False):
    extent = list(extent)
    n = int(np.prod(extent))
    out = np.zeros((n, n))
    check(abi.otvmc_lattice_couplings(len(extent), extent, J, alpha, kac, pbc, out))
    return out
