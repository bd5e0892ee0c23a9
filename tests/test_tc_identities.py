"""CPU checks of the algebra the tensor-core kernels rest on (no GPU): identities that turn a
sum over samples, sites or pairs into the products the kernels form, each checked against the
direct sum in FP64 or exact integers on small random inputs.

- Two-flip sums (the per-trajectory pair moments, LITF paragraph): with
  r_jk = r_j r_k exp(4 s_j s_k eta_jk) and u+- = r o [s = +-1], the three pair sums over j != k
  equal A1 + A2 + 2 A3, A1 + A2 - 2 A3 and A1 - A2 for A1 = u+ E+ u+, A2 = u- E+ u-,
  A3 = u+ E- u- (E+- = exp(+-4 eta), zero diagonal).
- The flip ratio's phase exp(-2 i s_j Im f_j) depends on Im f_j = Im a_j + sum_k Im eta_jk s_k
  only modulo pi, and s_k = +-1 lets every term be reduced modulo pi first.
- Balanced base-2^11 and base-16 digits recombine to the exact integer (wrapping 64-bit
  arithmetic), so digit-plane sums rebuild the exact integer sums.
"""
import numpy as np
import pytest

import synth


def _pair_sums_direct(r, s, eta):
    n = len(r)
    a = b = c = 0j
    for j in range(n):
        for k in range(n):
            if j == k:
                continue
            rjk = r[j] * r[k] * np.exp(4.0 * s[j] * s[k] * eta[j, k])
            a += rjk
            b += s[j] * s[k] * rjk
            c += s[k] * rjk
    return a, b, c


@pytest.mark.parametrize("n,seed", [(5, 1), (9, 2), (16, 3)])
def test_two_flip_sums_as_bilinear_forms(n, seed):
    g = synth.rng(seed)
    eta = g.normal(0, 0.2, (n, n)) + 1j * g.normal(0, 0.2, (n, n))
    eta = (eta + eta.T) / 2
    np.fill_diagonal(eta, 0.0)
    r = g.normal(0, 1, n) + 1j * g.normal(0, 1, n)
    s = np.where(g.random(n) < 0.5, 1.0, -1.0)
    Ep, Em = np.exp(4.0 * eta), np.exp(-4.0 * eta)
    np.fill_diagonal(Ep, 0.0)
    np.fill_diagonal(Em, 0.0)
    up, um = r * (s > 0), r * (s < 0)
    A1, A2, A3 = up @ Ep @ up, um @ Ep @ um, up @ Em @ um
    a, b, c = _pair_sums_direct(r, s, eta)
    scale = max(abs(a), abs(b), abs(c), 1.0)
    assert abs((A1 + A2 + 2 * A3) - a) < 1e-12 * scale
    assert abs((A1 + A2 - 2 * A3) - b) < 1e-12 * scale
    assert abs((A1 - A2) - c) < 1e-12 * scale


FX = 2.0 ** 48
FX_TWO_PI = 1768559438007110  # 2 pi in units of 2^-48, rounded to the nearest integer
FX_PI = FX_TWO_PI // 2


def _reduce_pi(q):
    """q (int) modulo FX_PI into [-FX_PI/2, FX_PI/2] (remainder truncated toward zero first)."""
    r = (abs(q) % FX_PI) * (1 if q >= 0 else -1)
    if r > FX_PI // 2:
        r -= FX_PI
    if r < -(FX_PI // 2):
        r += FX_PI
    return r


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_phase_depends_on_the_field_modulo_pi(seed):
    g = synth.rng(seed)
    n = 40
    q = [int(round(x * FX)) for x in g.normal(0, 3.0, n)]   # Im eta_jk in fixed point
    qa = int(round(g.normal(0, 3.0) * FX))                 # Im a_j
    s = [1 if x < 0.5 else -1 for x in g.random(n)]
    full = qa + sum(sk * qk for sk, qk in zip(s, q))
    red = _reduce_pi(qa) + sum(sk * _reduce_pi(qk) for sk, qk in zip(s, q))
    # the two differ by an integer multiple of FX_PI exactly
    assert (full - red) % FX_PI == 0
    for sj in (1, -1):
        # the ratio's phase -2 s_j Im f, in units where FX_TWO_PI is one turn, is the same
        assert (-2 * sj * full) % FX_TWO_PI == (-2 * sj * red) % FX_TWO_PI


def _balanced_digits(v, bits, count):
    base = 1 << bits
    half = base >> 1
    out = []
    for _ in range(count):
        d = ((v & (base - 1)) ^ half) - half
        out.append(d)
        v = (v - d) >> bits
    return out, v


# the estimator's Im entries reduced modulo pi and rounded to units of 2^-42 stay within
# FX_PI / 2^7 in magnitude, inside the range of four balanced base-2^11 digits
# (1023 (2^44 - 1) / 2047, about 0.9995 x 2^43); the D pass's quantised v stays below 2^62
@pytest.mark.parametrize("bits,count,limit", [(11, 4, (FX_PI // 2 >> 6) + 1), (4, 16, 1 << 62)])
def test_balanced_digits_recombine_exactly(bits, count, limit):
    g = synth.rng(7)
    vals = [int(x) for x in g.integers(-limit, limit, 2000)] + [limit - 1, -limit, 0, 1, -1]
    half = 1 << (bits - 1)
    for v in vals:
        ds, rest = _balanced_digits(v, bits, count)
        assert all(-half <= d < half for d in ds)
        assert rest == 0
        assert sum(d << (bits * p) for p, d in enumerate(ds)) == v


def test_digit_plane_sums_rebuild_the_integer_sum():
    """Sums over samples of O_k(x) times each digit plane of q(x), recombined, give sum_x O_k q
    exactly (the D pass: sixteen base-16 digits of 64-bit q), even where 64-bit q wraps."""
    g = synth.rng(8)
    ns = 500
    q = [int(x) for x in g.integers(-(1 << 62), 1 << 62, ns)]
    o = [1 if x < 0.5 else -1 for x in g.random(ns)]
    planes = [_balanced_digits(v, 4, 16)[0] for v in q]
    sums = [sum(o[x] * planes[x][p] for x in range(ns)) for p in range(16)]
    assert all(abs(sp) <= 8 * ns for sp in sums)
    rebuilt = sum(sp << (4 * p) for p, sp in enumerate(sums)) & ((1 << 64) - 1)
    want = sum(ox * qx for ox, qx in zip(o, q)) & ((1 << 64) - 1)
    assert rebuilt == want
