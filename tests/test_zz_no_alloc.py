"""The allocation-free local estimators (for callers that cannot hand the library scratch
memory: device memory owned by a manager with a hard budget, or a loop that cannot afford an
allocation's device synchronisation) must give what the workspace version gives, bit for bit,
call after call, although every call reuses the same fixed scratch array inside the library.

This file is collected last on purpose, so that a run that stops at its first failure has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from gpu_helpers import Case, require_gpu, from_dev_complex, torch
import synth
from paper_2506_23928_gb300 import abi
from paper_2506_23928_gb300.abi import check

pytestmark = pytest.mark.gpu
FP64, MIXED = abi.OTVMC_PREC_FP64, abi.OTVMC_PREC_MIXED


def _run(c, precision, th_d, sp, dW_d, T, ns, dt, noalloc):
    E = torch.zeros((T, ns, 2), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(E)
    lpl = torch.zeros((T, max(c.nops, 1)), dtype=torch.float64, device="cuda")
    if noalloc:
        status = torch.zeros(2, dtype=torch.int32, device="cuda")  # error code, then its detail
        check(abi.otvmc_local_estimators_noalloc(c.ans.handle, th_d, sp, T, ns, dW_d, dt, precision, E, v, lpl,
                                                 status))
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [0, 0]
    else:
        work, nb = c.work(T, ns, precision)
        check(abi.otvmc_local_estimators(c.ans.handle, th_d, sp, T, ns, dW_d, dt, precision, E, v, lpl, work, nb))
        check(abi.otvmc_check(work))
    return from_dev_complex(E)[..., 0], from_dev_complex(v)[..., 0], lpl.cpu().numpy()


def test_local_estimators_noalloc_matches_workspace_version_on_consecutive_calls():
    require_gpu()
    c = Case((24,), h=0.7, kappa=0.1, gamma=0.05)
    dt = 0.01
    # two calls in a row with different batch shapes and inputs: the second one reuses the
    # scratch the first one left behind; the same kernels on the same inputs give the same bits
    for seed, T, ns in ((101, 3, 500), (202, 5, 333)):
        th, th_d = c.theta(seed, T, 0.1)
        sig, sp = c.spins(seed + 1, T, ns)
        dW_d = torch.from_numpy(synth.random_normals(seed + 2, (T, c.nops), np.sqrt(dt))).cuda()
        for precision in (FP64, MIXED):
            ref = _run(c, precision, th_d, sp, dW_d, T, ns, dt, noalloc=False)
            got = _run(c, precision, th_d, sp, dW_d, T, ns, dt, noalloc=True)
            for g, r in zip(got, ref):
                assert np.array_equal(g, r)


def test_local_estimators_noalloc_reports_device_errors_in_both_status_words():
    """A parameter field beyond the fixed-point range on trajectory 1 is reported as
    OTVMC_ERR_RANGE with that trajectory in the second word; the next call with valid
    parameters succeeds."""
    require_gpu()
    c = Case((16,), kappa=0.1)
    T, ns, dt = 3, 64, 0.01
    th, _ = c.theta(5, T, 0.1)
    bad = th.copy()
    bad[1, 0] = 1.0e4  # |a_0| above the fixed-point range of the fields
    from gpu_helpers import to_dev_complex
    sig, sp = c.spins(6, T, ns)
    dW_d = torch.zeros((T, c.nops), dtype=torch.float64, device="cuda")
    v = torch.zeros((T, ns, 2), dtype=torch.float64, device="cuda")
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    check(abi.otvmc_local_estimators_noalloc(c.ans.handle, to_dev_complex(bad), sp, T, ns, dW_d, dt, MIXED, None, v,
                                             None, status))
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [abi.OTVMC_ERR_RANGE, 1]
    status.zero_()
    check(abi.otvmc_local_estimators_noalloc(c.ans.handle, to_dev_complex(th), sp, T, ns, dW_d, dt, MIXED, None, v,
                                             None, status))
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0, 0]


def test_local_estimators_noalloc_rejects_batches_beyond_its_scratch():
    require_gpu()
    c = Case((64,), kappa=0.1)
    th, th_d = c.theta(7, 1, 0.1)
    sig, sp = c.spins(8, 1, 64)
    v = torch.zeros((1, 64, 2), dtype=torch.float64, device="cuda")
    dW_d = torch.zeros((1, c.nops), dtype=torch.float64, device="cuda")
    # 8 trajectories x 4096 samples x 64 sites need ~37 MB of scratch: rejected before any launch
    st = abi.otvmc_local_estimators_noalloc(c.ans.handle, th_d, sp, 8, 4096, dW_d, 0.01, MIXED, None, v, None, None)
    assert st == abi.OTVMC_ERR_WORKSPACE
    assert "scratch" in abi.otvmc_last_error()
