"""The C ABI library without a GPU: it builds, loads, exports every declared entry point,
and its host-only helpers agree with the oracle."""
import os
import re

import numpy as np
import pytest

import paper_2506_23928_gb300 as pkg
from paper_2506_23928_gb300 import abi, build
from oracle.model import couplings
from oracle.observables import squeezing, ensemble

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "otvmc.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"OTVMC_API\s+[\w\s\*]*?\b(otvmc_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["otvmc_model_create", "otvmc_ansatz_create", "otvmc_sample", "otvmc_local_estimators",
                     "otvmc_build_S_F", "otvmc_solve_step", "otvmc_run_trajectories", "otvmc_observables"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(abi.SIGNATURES)


def test_binding_constants_match_header():
    """Every enum value the header defines and the binding names has the header's value."""
    text = open(HEADER).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(OTVMC_\w+)\s*=\s*(\d+)", text)}
    named = [k for k in consts if hasattr(abi, k)]
    assert len(named) >= 20
    for k in named:
        assert getattr(abi, k) == consts[k], k
    for k in ("OTVMC_PROFILE_OFF", "OTVMC_PROFILE_ON", "OTVMC_PROFILE_SERIAL", "OTVMC_RBM_T_FACTORED"):
        assert k in named
    # kernel classes: the binding lists one name per class, in the header's order
    classes = sorted((v, k) for k, v in consts.items() if k.startswith("OTVMC_K_") and k != "OTVMC_K_CLASSES")
    assert [v for v, _ in classes] == list(range(consts["OTVMC_K_CLASSES"]))
    assert len(abi.KERNEL_CLASSES) == consts["OTVMC_K_CLASSES"]


@pytest.mark.parametrize("extent,alpha,kac,pbc", [((8,), 1.5, False, False), ((10,), 1.0, True, True),
                                                   ((4, 5), 3.0, False, False), ((4, 4), 1.5, False, True)])
def test_lattice_couplings_match_oracle(lib, extent, alpha, kac, pbc):
    got = pkg.lattice_couplings(extent, 1.3, alpha, kac, pbc)
    want = couplings(extent, 1.3, alpha, kac=kac, pbc=pbc)
    assert np.allclose(got, want, rtol=1e-14, atol=0)


def test_ensemble_helper_matches_oracle(lib):
    g = np.random.default_rng(3)
    nt, n = 40, 12
    m = g.normal(0, 0.1, (nt, 3)) + np.array([0.7, 0.1, -0.2])
    q = np.zeros((nt, 3, 3))
    for t in range(nt):
        A = g.normal(0, 0.05, (3, 3))
        q[t] = A @ A.T + np.outer(m[t], m[t])
    mom = np.concatenate([m, q[:, [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]], axis=1)
    M, C, xi2, dM = np.zeros(3), np.zeros(9), np.zeros(1), np.zeros(3)
    abi.check(abi.otvmc_ensemble(np.ascontiguousarray(mom), nt, n, M, C, xi2, dM))
    M0, C0, dM0 = ensemble(m, q)
    assert np.allclose(M, M0, atol=1e-14)
    assert np.allclose(C.reshape(3, 3), C0, atol=1e-14)
    assert np.allclose(dM, dM0, atol=1e-14)
    assert abs(xi2[0] - squeezing(M0, C0, n)) < 1e-12


def test_weighted_ensemble_helper_matches_oracle(lib):
    """The linear SSE's average (each trajectory's moments weighted by its norm Q_j, App. B)."""
    from oracle.observables import ensemble_weighted
    g = np.random.default_rng(5)
    nt, n = 30, 10
    m = g.normal(0, 0.1, (nt, 3)) + np.array([0.6, 0.2, -0.3])
    q = np.zeros((nt, 3, 3))
    for t in range(nt):
        A = g.normal(0, 0.05, (3, 3))
        q[t] = A @ A.T + np.outer(m[t], m[t])
    Q = np.exp(g.normal(0, 0.3, nt))
    mom = np.concatenate([m, q[:, [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]], axis=1)
    M, C, xi2, dM = np.zeros(3), np.zeros(9), np.zeros(1), np.zeros(3)
    abi.check(abi.otvmc_ensemble_weighted(np.ascontiguousarray(mom), Q, nt, n, M, C, xi2, dM))
    M0, C0, dM0 = ensemble_weighted(m, q, Q)
    assert np.allclose(M, M0, atol=1e-14)
    assert np.allclose(C.reshape(3, 3), C0, atol=1e-14)
    assert np.allclose(dM, dM0, atol=1e-14)
    assert abs(xi2[0] - squeezing(M0, C0, n)) < 1e-12


def test_bad_arguments_are_rejected_without_a_gpu(lib):
    out = np.zeros(4)
    st = abi.otvmc_lattice_couplings(3, [2, 2, 1], 1.0, 1.0, 0, 0, out)
    assert st == abi.OTVMC_ERR_INVALID
    assert "dim" in abi.otvmc_last_error()
