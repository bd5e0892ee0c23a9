"""The bounded waits of the tensor-core kernels (Gram, Cholesky update and panel): with the
wait limit lowered far below the time a copy takes, the kernels give up, drain what they have
in flight, record OTVMC_ERR_TIMEOUT and return, and the context stays usable: the next calls
with the normal limit give the results of calls made before, bit for bit."""
import numpy as np
import pytest

from gpu_helpers import Case, require_gpu, to_dev_complex, torch
import synth
from paper_2506_23928_gb300 import abi
from paper_2506_23928_gb300.abi import check

pytestmark = pytest.mark.gpu
MIXED = abi.OTVMC_PREC_MIXED


def _build(c, sp, v_d, T, ns, work, nb):
    P = c.P
    G = torch.zeros((T, P, P), dtype=torch.float32, device="cuda")
    ob = torch.zeros((T, P), dtype=torch.float64, device="cuda")
    D = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    check(abi.otvmc_build_S_F(c.ans.handle, None, sp, v_d, T, ns, MIXED, None, G, ob, D, work, nb))
    return G, ob, D


def _solve(c, T, ns, G, ob, D, work, nb):
    delta = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    check(abi.otvmc_solve_step(c.ans.handle, T, ns, MIXED, abi.OTVMC_REG_SHIFT, 1e-3, 4.0, None, G, ob, D, delta,
                               None, work, nb))
    return delta


def test_wait_timeout_is_reported_and_the_next_call_succeeds():
    require_gpu()
    c = Case((64,), kappa=0.1)
    T, ns = 2, 4096
    sig, sp = c.spins(3, T, ns)
    v = synth.random_normals(4, (T, ns)) + 1j * synth.random_normals(5, (T, ns))
    v_d = to_dev_complex(v)
    work, nb = c.work(T, ns, MIXED)
    G0, ob0, D0 = _build(c, sp, v_d, T, ns, work, nb)
    assert abi.otvmc_check(work) == abi.OTVMC_OK
    d0 = _solve(c, T, ns, G0, ob0, D0, work, nb)
    assert abi.otvmc_check(work) == abi.OTVMC_OK
    check(abi.otvmc_debug_set_wait_limit(1))  # 1 ns: every pipeline wait that has to wait gives up
    try:
        _build(c, sp, v_d, T, ns, work, nb)
        assert abi.otvmc_check(work) == abi.OTVMC_ERR_TIMEOUT
        _solve(c, T, ns, G0, ob0, D0, work, nb)  # valid inputs: only the waits make it fail
        assert abi.otvmc_check(work) == abi.OTVMC_ERR_TIMEOUT
    finally:
        check(abi.otvmc_debug_set_wait_limit(0))
    G1, ob1, D1 = _build(c, sp, v_d, T, ns, work, nb)
    assert abi.otvmc_check(work) == abi.OTVMC_OK
    d1 = _solve(c, T, ns, G1, ob1, D1, work, nb)
    assert abi.otvmc_check(work) == abi.OTVMC_OK
    for a, b in ((G0, G1), (ob0, ob1), (D0, D1), (d0, d1)):
        assert torch.equal(a, b)
