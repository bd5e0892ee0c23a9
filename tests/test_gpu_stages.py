"""Parity of every stage of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative to the largest expected magnitude): FP64 path 1e-10; mixed path
1e-5 on E_eff, v, S, D and observables, 1e-4 on the parameter update delta.  Integer
work (chains, spin words) is compared bit for bit.
"""
import numpy as np
import pytest

from gpu_helpers import Case, require_gpu, to_dev_complex, from_dev_complex, unpack, rel_err, torch
import synth
from oracle import philox, tvmc
from oracle.observables import moments_from_samples
from paper_2506_23928_gb300 import abi
from paper_2506_23928_gb300.abi import check

pytestmark = pytest.mark.gpu
FP64, MIXED = abi.OTVMC_PREC_FP64, abi.OTVMC_PREC_MIXED
TOL = {FP64: 1e-10, MIXED: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_noise_matches_oracle():
    c = Case((20,), kappa=0.1, gamma=0.05)
    dW = torch.zeros((5, c.nops), dtype=torch.float64, device="cuda")
    check(abi.otvmc_draw_noise(c.model.handle, 5, 3, 1234567, 7, 0.005, dW))
    torch.cuda.synchronize()
    want = philox.wiener_increments(1234567, np.arange(3, 8), 7, c.nops, 0.005)
    assert rel_err(dW.cpu().numpy(), want) < 1e-14


@pytest.mark.parametrize("n", [5, 70, 130])
def test_init_chains_bit_exact(n):
    c = Case((n,))
    ns, T = 300, 2
    sp = torch.zeros((T, ns, c.W), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(c.ans.handle, T, 1, ns, 99, sp))
    got = unpack(sp, n)
    for t in range(T):
        assert np.array_equal(got[t], philox.initial_spins(99, 1 + t, ns, n))
    words = sp.cpu().numpy().view(np.uint64)
    if n % 64:
        assert np.all(words[..., -1] >> np.uint64(n % 64) == 0)


@pytest.mark.parametrize("n,ns", [(8, 200), (13, 77), (37, 160), (70, 96)])
def test_sample_bit_exact(n, ns):
    c = Case((n,), kappa=0.1)
    T, traj0, seed, ev, sweeps = 2, 5, 2024, 11, 2
    th, th_d = c.theta(3, T, 0.15)
    sig, sp = c.spins(4, T, ns)
    acc = torch.zeros(T, dtype=torch.int64, device="cuda")
    work, nb = c.work(T, ns, FP64)
    check(abi.otvmc_sample(c.ans.handle, th_d, T, traj0, ns, sweeps, seed, ev, sp, acc, work, nb))
    check(abi.otvmc_check(work))
    got = unpack(sp, n)
    for t in range(T):
        want, a = tvmc.metropolis(c.oans, th[t], sig[t], seed, traj0 + t, ev, sweeps)
        assert np.array_equal(got[t], want)
        assert int(acc[t]) == int(a.sum())


def _estimators(c, precision, T, ns, dt=0.01, scale=0.1):
    th, th_d = c.theta(11, T, scale)
    sig, sp = c.spins(12, T, ns)
    dW = synth.random_normals(13, (T, c.nops), np.sqrt(dt))
    dW_d = torch.from_numpy(dW).cuda()
    E = torch.zeros((T, ns, 2), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(E)
    lpl = torch.zeros((T, max(c.nops, 1)), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, precision)
    check(abi.otvmc_local_estimators(c.ans.handle, th_d, sp, T, ns, dW_d, dt, precision, E, v, lpl, work, nb))
    check(abi.otvmc_check(work))
    return th, sig, dW, from_dev_complex(E)[..., 0], from_dev_complex(v)[..., 0], lpl.cpu().numpy()


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,ns", [(12, 500), (33, 130)])
def test_local_estimators(precision, n, ns):
    c = Case((n,), h=0.7, kappa=0.1, gamma=0.05)
    T, dt = 3, 0.01
    th, sig, dW, E, v, lpl = _estimators(c, precision, T, ns, dt)
    for t in range(T):
        ev = tvmc.evaluate(c.omodel, c.oans, th[t], sig[t], tvmc.mc_weights(ns), dW[t], dt)
        assert rel_err(E[t], ev["E"]) < TOL[precision]
        assert rel_err(v[t], tvmc.local_v(ev, dW[t], dt)) < TOL[precision]
        assert rel_err(lpl[t, :c.nops], ev["lpl"]) < TOL[precision]


@pytest.mark.parametrize("n,ns,scale", [(64, 1100, 0.1), (100, 300, 0.1), (128, 260, 0.05), (64, 700, 0.6),
                                         (150, 200, 0.05)])
def test_local_estimators_large_n(n, ns, scale):
    """The mixed path's estimators at N = 64, 100 and 128 run on the tensor cores (one or two
    64-site blocks of the contraction, ragged site blocks of 16 and sample tiles of 128); N = 150
    on the SIMT kernel.  Scale 0.6 makes |Im f_j| several times pi, so that the fixed-point
    reduction of the phase is exercised.  E_eff, v and <L + L^+> against the oracle."""
    c = Case((n,), h=0.7, kappa=0.1, gamma=0.05)
    T, dt = 2, 0.01
    th, sig, dW, E, v, lpl = _estimators(c, MIXED, T, ns, dt, scale)
    for t in range(T):
        ev = tvmc.evaluate(c.omodel, c.oans, th[t], sig[t], tvmc.mc_weights(ns), dW[t], dt, with_S=False)
        assert rel_err(E[t], ev["E"]) < TOL[MIXED]
        assert rel_err(v[t], tvmc.local_v(ev, dW[t], dt)) < TOL[MIXED]
        assert rel_err(lpl[t, :c.nops], ev["lpl"]) < TOL[MIXED]


def _build(c, precision, T, ns, v, sp, want_S=True):
    v_d = to_dev_complex(v)
    P = c.P
    S = torch.zeros((T, P, P), dtype=torch.float64, device="cuda") if want_S else None
    G = torch.zeros((T, P, P), dtype=torch.float32, device="cuda") if precision == MIXED else None
    ob = torch.zeros((T, P), dtype=torch.float64, device="cuda")
    D = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, precision)
    check(abi.otvmc_build_S_F(c.ans.handle, None, sp, v_d, T, ns, precision, S, G, ob, D, work, nb))
    check(abi.otvmc_check(work))
    return S, G, ob, D


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,ns", [(20, 1000), (6, 64)])
def test_build_S_F(precision, n, ns):
    c = Case((n,), h=0.7, kappa=0.1, gamma=0.05)
    T, dt = 2, 0.01
    th, _ = c.theta(21, T, 0.1)
    sig, sp = c.spins(22, T, ns)
    dW = synth.random_normals(23, (T, c.nops), np.sqrt(dt))
    evs = [tvmc.evaluate(c.omodel, c.oans, th[t], sig[t], tvmc.mc_weights(ns), dW[t], dt) for t in range(T)]
    v = np.stack([tvmc.local_v(evs[t], dW[t], dt) for t in range(T)])
    S, G, ob, D = _build(c, precision, T, ns, v, sp)
    S, D = S.cpu().numpy(), from_dev_complex(D)[..., 0]
    for t in range(T):
        assert rel_err(S[t], evs[t]["S"].real) < 1e-12
        assert rel_err(D[t], evs[t]["D"]) < 1e-10
        assert rel_err(ob.cpu().numpy()[t], evs[t]["O"].real.mean(axis=0)) < 1e-14
    if precision == MIXED:
        Gn = G.cpu().numpy()
        for t in range(T):
            O = evs[t]["O"].real
            iu = np.triu_indices(c.P)
            assert np.array_equal(Gn[t][iu], (O.T @ O)[iu])


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_build_S_F_many_tiles(precision):
    """P = 2080 (N = 64): 17 x 9 tiles of the Gram kernel with ragged edges."""
    c = Case((64,), kappa=0.1, gamma=0.05)
    T, ns, dt = 2, 520, 0.005
    th, _ = c.theta(31, T, 0.05)
    sig, sp = c.spins(32, T, ns)
    dW = synth.random_normals(33, (T, c.nops), np.sqrt(dt))
    evs = [tvmc.evaluate(c.omodel, c.oans, th[t], sig[t], tvmc.mc_weights(ns), dW[t], dt) for t in range(T)]
    v = np.stack([tvmc.local_v(evs[t], dW[t], dt) for t in range(T)])
    S, G, ob, D = _build(c, precision, T, ns, v, sp)
    S, D = S.cpu().numpy(), from_dev_complex(D)[..., 0]
    for t in range(T):
        assert rel_err(S[t], evs[t]["S"].real) < 1e-12
        assert rel_err(D[t], evs[t]["D"]) < 1e-10


@pytest.mark.parametrize("n,ns", [(22, 136), (22, 4096), (64, 4096)])
def test_D_from_gram_pass(n, ns):
    """On the mixed path D and obar come out of the Gram kernel: the quantised centred v enters as
    extra rows of O (balanced base-16 digits, exact in E4M3, digit sums exact in FP32) and a row
    of ones.  P = 253 needs one more column tile for those rows, P = 2080 has room in its last
    tile.  obar equals the FP64 path's (exact counts) bit for bit, D agrees with the FP64 path's
    GEMV to rounding (a digit lost or misplaced would show at 1e-10 or above), and G stays the
    exact count matrix."""
    c = Case((n,), h=0.7, kappa=0.1, gamma=0.05)
    T = 3
    sig, sp = c.spins(41, T, ns)
    g = synth.rng(42)
    v = g.normal(0, 1, (T, ns)) + 1j * g.normal(0, 1, (T, ns))
    _, G, ob_m, D_m = _build(c, MIXED, T, ns, v, sp, want_S=False)
    _, _, ob_f, D_f = _build(c, FP64, T, ns, v, sp)
    assert torch.equal(ob_m, ob_f)
    D_m, D_f = from_dev_complex(D_m)[..., 0], from_dev_complex(D_f)[..., 0]
    for t in range(T):
        assert rel_err(D_m[t], D_f[t]) < 1e-13
    O = np.concatenate([sig[0].astype(np.float64), np.stack([sig[0][:, j] * sig[0][:, k] for j in range(n)
                                                             for k in range(j + 1, n)], axis=1)], axis=1)
    iu = np.triu_indices(c.P)
    assert np.array_equal(G.cpu().numpy()[0][iu], (O.T @ O)[iu])


@pytest.mark.parametrize("ns", [1 << 17, 131064])
def test_gram_accumulation_at_the_largest_sums(ns):
    """The FP8 Gram pass at its largest sums: ns = 2^17 samples (the most that take D from the
    Gram pass) and a ragged count just below it.  Site 0 follows the sign of v and site 1 is up
    in three samples of four, so the digit sums of q against O_0 approach 8 ns = 2^20 and the
    counts G_00 = ns, G_01 ~ ns / 2 stay large while the products added to them are +-1: a
    tensor-core accumulation narrower than FP32 would drop units here.  G must equal the
    exact integer Gram and D the FP64 path's to rounding."""
    n = 6
    c = Case((n,), h=0.7, kappa=0.1, gamma=0.05)
    g = synth.rng(51)
    re = np.where(g.random(ns) < 0.5, -1.0, 1.0) * (1.0 + 0.01 * g.random(ns))
    v = (re + 1j * 0.5 * re)[None, :]
    sig = synth.random_spins(52, 1, ns, n)
    sig[0, :, 0] = np.where(re > 0, 1, -1)
    sig[0, :, 1] = np.where(g.random(ns) < 0.75, 1, -1)
    sp = torch.from_numpy(synth.pack_spins(sig).view(np.int64)).cuda()
    _, G, ob_m, D_m = _build(c, MIXED, 1, ns, v, sp, want_S=False)
    _, _, ob_f, D_f = _build(c, FP64, 1, ns, v, sp)
    assert torch.equal(ob_m, ob_f)
    assert rel_err(from_dev_complex(D_m)[0, :, 0], from_dev_complex(D_f)[0, :, 0]) < 1e-13
    s0 = sig[0].astype(np.float64)
    O = np.concatenate([s0, np.stack([s0[:, j] * s0[:, k] for j in range(n) for k in range(j + 1, n)], axis=1)],
                       axis=1)
    iu = np.triu_indices(c.P)
    assert np.array_equal(G.cpu().numpy()[0][iu], (O.T @ O)[iu])


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_solve_step(precision):
    c = Case((16,), kappa=0.1, gamma=0.05)
    T, ns, dt, eps = 3, 600, 0.01, 1e-4
    th, _ = c.theta(41, T, 0.1)
    sig, sp = c.spins(42, T, ns)
    dW = synth.random_normals(43, (T, c.nops), np.sqrt(dt))
    evs = [tvmc.evaluate(c.omodel, c.oans, th[t], sig[t], tvmc.mc_weights(ns), dW[t], dt) for t in range(T)]
    v = np.stack([tvmc.local_v(evs[t], dW[t], dt) for t in range(T)])
    S, G, ob, D = _build(c, precision, T, ns, v, sp, want_S=(precision == FP64))
    delta = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    shift = torch.zeros(T, dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, precision)
    check(abi.otvmc_solve_step(c.ans.handle, T, ns, precision, abi.OTVMC_REG_SHIFT, eps, 4.0, S, G, ob, D, delta,
                               shift, work, nb))
    check(abi.otvmc_check(work))
    got = from_dev_complex(delta)[..., 0]
    tol = 1e-10 if precision == FP64 else 1e-4
    for t in range(T):
        want = tvmc.solve_shift(evs[t]["S"], evs[t]["D"], eps)
        assert rel_err(got[t], want) < tol
        assert float(shift[t]) == eps


def test_solve_step_fp64_from_oracle_S():
    """The FP64 solve alone, with S and D given by the oracle."""
    c = Case((24,), kappa=0.1)
    T, ns, eps = 2, 400, 1e-3
    th, _ = c.theta(51, T, 0.1)
    sig, _ = c.spins(52, T, ns)
    evs = [tvmc.evaluate(c.omodel, c.oans, th[t], sig[t], tvmc.mc_weights(ns), np.zeros(c.nops), 0.02)
           for t in range(T)]
    S = torch.from_numpy(np.stack([e["S"].real for e in evs])).cuda()
    D = to_dev_complex(np.stack([e["D"] for e in evs]))
    delta = torch.zeros((T, c.P, 2), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, FP64)
    check(abi.otvmc_solve_step(c.ans.handle, T, ns, FP64, abi.OTVMC_REG_SHIFT, eps, 4.0, S, None, None, D, delta,
                               None, work, nb))
    check(abi.otvmc_check(work))
    got = from_dev_complex(delta)[..., 0]
    for t in range(T):
        assert rel_err(got[t], tvmc.solve_shift(evs[t]["S"], evs[t]["D"], eps)) < 1e-10


def test_solve_not_positive_definite_reports_status():
    c = Case((4,), kappa=0.1)
    T, P = 1, c.P
    # shift retries raise eps to at most 1e-4 * 1e6 = 100, which cannot rescue -1000 I
    S = -1000.0 * torch.eye(P, dtype=torch.float64, device="cuda")[None].contiguous()
    D = torch.ones((T, P, 2), dtype=torch.float64, device="cuda")
    delta = torch.full((T, P, 2), 7.0, dtype=torch.float64, device="cuda")
    work, nb = c.work(T, 8, FP64)
    check(abi.otvmc_solve_step(c.ans.handle, T, 8, FP64, abi.OTVMC_REG_SHIFT, 1e-4, 4.0, S, None, None, D, delta,
                               None, work, nb))
    assert abi.otvmc_check(work) == abi.OTVMC_ERR_NOT_PD
    assert torch.all(delta == 0)
    assert abi.otvmc_check(work) == abi.OTVMC_OK  # cleared


@pytest.mark.parametrize("scheme", [abi.OTVMC_HEUN, abi.OTVMC_MIDPOINT])
def test_sde_combine(scheme):
    T, P = 3, 50
    g = np.random.default_rng(5)
    th, d0, d1 = [g.normal(size=(T, P)) + 1j * g.normal(size=(T, P)) for _ in range(3)]
    d1[1, 7] = np.nan
    work = torch.zeros(256, dtype=torch.uint8, device="cuda")
    out0 = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    out1 = torch.zeros_like(out0)
    failed = torch.zeros(T, dtype=torch.int32, device="cuda")
    args = [to_dev_complex(x) for x in (th, d0, d1)]
    check(abi.otvmc_sde_combine(T, P, scheme, 0, args[0], args[1], None, out0, None, work, 256))
    check(abi.otvmc_sde_combine(T, P, scheme, 1, args[0], args[1], args[2], out1, failed, work, 256))
    assert abi.otvmc_check(work) == abi.OTVMC_ERR_NONFINITE
    c = 1.0 if scheme == abi.OTVMC_HEUN else 0.5
    assert rel_err(from_dev_complex(out0)[..., 0], th + c * d0) < 1e-15
    want = th + 0.5 * (d0 + d1) if scheme == abi.OTVMC_HEUN else th + d1
    got = from_dev_complex(out1)[..., 0]
    assert rel_err(got[[0, 2]], want[[0, 2]]) < 1e-15
    assert np.array_equal(got[1], th[1])
    assert failed.cpu().tolist() == [0, 1, 0]


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,ns", [(10, 400), (3, 33), (40, 64), (64, 1100), (33, 700)])
def test_observables(precision, n, ns):
    """Moments against the oracle; on the mixed path N = 33 ... 64 take the tensor-core kernel
    (one ragged tile, several tiles and CTAs), the others the SIMT kernel."""
    c = Case((n,), kappa=0.1)
    T = 3
    th, th_d = c.theta(61, T, 0.2)
    sig, sp = c.spins(62, T, ns)
    mom = torch.zeros((T, 9), dtype=torch.float64, device="cuda")
    work, nb = c.work(T, ns, precision)
    check(abi.otvmc_observables(c.ans.handle, th_d, sp, T, ns, precision, mom, work, nb))
    check(abi.otvmc_check(work))
    got = mom.cpu().numpy()
    for t in range(T):
        m, q = moments_from_samples(c.oans, th[t], sig[t], tvmc.mc_weights(ns))
        want = np.concatenate([m, q[[0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]]])
        assert rel_err(got[t], want) < TOL[precision]


def test_argument_errors():
    c = Case((6,))
    work, nb = c.work(1, 64, MIXED)
    v = torch.zeros((1, 60, 2), dtype=torch.float64, device="cuda")
    sp = torch.zeros((1, 60, 1), dtype=torch.int64, device="cuda")
    G = torch.zeros((1, c.P, c.P), dtype=torch.float32, device="cuda")
    D = torch.zeros((1, c.P, 2), dtype=torch.float64, device="cuda")
    st = abi.otvmc_build_S_F(c.ans.handle, None, sp, v, 1, 60, MIXED, None, G, None, D, work, nb)
    assert st == abi.OTVMC_ERR_INVALID  # ns % 8 != 0 for the tensor-core path
    st = abi.otvmc_build_S_F(c.ans.handle, None, sp, v, 1, 64, MIXED, None, G, None, D, work, 1024)
    assert st == abi.OTVMC_ERR_WORKSPACE
