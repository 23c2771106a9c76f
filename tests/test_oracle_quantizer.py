"""Pins for the oracle's error-bounded residual quantizer (Stage 4).

The quantizer is defined as q = round-half-even((x - xhat) / Delta) on the
exact real difference, Delta = 2^floor(log2(2 alpha e)), e = tau max(x).
These tests check the oracle against exact rational arithmetic (Python
``fractions.Fraction``), constructed exact and near ties, and the pointwise
bound |x' - x| <= Delta / 2 (+ half an ulp of x').
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2212_10733_gb300 import synth


def exact_q(x: float, xh: float, dl: float) -> int:
    # Python's round() on a Fraction rounds half to even
    return round((Fraction(x) - Fraction(float(np.float32(xh)))) / Fraction(dl))


def exact_code(x: float, xh: float, dl: float):
    """Nearest reconstruction level among xh + q dl (|q| <= 32766, q the
    round-half-even index) and 0, in exact rational arithmetic; ties keep the
    grid level.  Returns (code, x')."""
    xh = float(np.float32(xh))
    if not np.isfinite(xh):
        return oracle.ESCAPE, x
    q = exact_q(x, xh, dl)
    if abs(q) > oracle.CODE_MAX:
        return oracle.ESCAPE, x
    g = Fraction(xh) + q * Fraction(dl)
    if abs(Fraction(x)) < abs(Fraction(x) - g):
        return oracle.ZERO_CODE, 0.0
    return q, float(g)  # float() of a Fraction rounds to nearest even


def test_delta_is_power_of_two_below_budget():
    rng = np.random.default_rng(1)
    for e in np.exp(rng.uniform(-40, 40, size=2000)):
        for alpha in (0.5, 0.125, 0.3):
            dl = oracle.delta(e, alpha)
            m, E = math.frexp(dl)
            assert m == 0.5  # exact power of two
            budget = Fraction(2.0 * alpha * e)  # 2 alpha e as computed in FP64
            assert Fraction(dl) <= budget < 2 * Fraction(dl)


def test_round_residual_random_vs_fraction():
    rng = np.random.default_rng(2)
    n = 20000
    x = np.exp(rng.uniform(-30, 5, size=n))
    xh = (x * (1 + rng.normal(0, 1e-2, size=n))).astype(np.float32)
    dls = 2.0 ** rng.integers(-40, 0, size=n)
    for a, b, d in zip(x, xh, dls):
        q = oracle.round_residual(float(a), float(b), float(d))
        qe = exact_q(float(a), float(b), float(d))
        assert q == qe, (a, b, d, q, qe)


def test_round_residual_exact_ties_go_to_even():
    dl = 2.0 ** -14
    for m in range(-40, 41):
        xh = np.float32(0.75)
        x = float(xh) + (m + 0.5) * dl  # exactly representable
        q = oracle.round_residual(x, float(xh), dl)
        assert Fraction(x) - Fraction(float(xh)) == (m + Fraction(1, 2)) * Fraction(dl)
        assert q == exact_q(x, float(xh), dl)
        assert int(q) % 2 == 0


def test_round_residual_near_ties_use_the_lost_bits():
    # fl(x - xhat) lands exactly on a tie although the exact difference does not:
    # x = (m + 1/2) Delta and xhat a float far below half an ulp of x.
    dl = 2.0 ** -10
    for m in range(1, 200):
        x = (m + 0.5) * dl
        for xh in (1e-30, -1e-30, 3e-38, -3e-38):
            xh32 = float(np.float32(xh))
            assert x - xh32 == x  # the subtraction rounds onto the tie
            q = oracle.round_residual(x, xh32, dl)
            qe = exact_q(x, xh32, dl)
            assert q == qe
            assert qe == (m if xh32 > 0 else m + 1)


def test_quantize_matches_fraction_and_bound(grid):
    n = 24
    x = synth.histograms(n, synth.config_seed(0))
    xh = synth.stand_in_xhat(x, 5)
    tau = 1e-4
    codes, xp, scale, dl, st = oracle.quantize(x, xh, tau)
    assert np.all(scale == x.max(axis=1))
    for b in range(n):
        assert dl[b] == oracle.delta(tau * scale[b], 0.5)
        for p in range(0, synth.P, 3):
            ce, ve = exact_code(x[b, p], xh[b, p], dl[b])
            assert codes[b, p] == ce and xp[b, p] == ve, (b, p)
        ulp = np.spacing(np.abs(xp[b]))
        assert np.all(np.abs(xp[b] - x[b]) <= dl[b] / 2 + ulp)
        assert np.all(xp[b] >= 0.0)
    assert np.any(codes == oracle.ZERO_CODE)
    assert np.all((st & oracle.VERBATIM) == 0)
    # with 1% + 0.2% noise most histograms need codes
    assert np.mean(codes != 0) > 0.5


def test_quantize_escapes_and_special_images():
    x = synth.histograms(4, synth.config_seed(0))
    xh = synth.stand_in_xhat(x, 6)
    xh[0, 10] = np.nan
    xh[0, 11] = np.inf
    xh[0, 12] = 1e30
    x[1, 5] = -1.0  # negative input: not a histogram
    x[2, :] = 0.0  # all-zero image
    x[3, 7] = np.nan
    codes, xp, scale, dl, st = oracle.quantize(x, xh, 1e-4)
    assert list(codes[0, 10:13]) == [oracle.ESCAPE] * 3
    assert np.all(xp[0, 10:13] == x[0, 10:13])
    assert st[0] & oracle.CODE_ESCAPE
    assert st[1] & oracle.VERBATIM and st[1] & oracle.NONFINITE_INPUT
    assert np.all(codes[1] == oracle.ESCAPE)
    assert st[2] & oracle.ZERO_IMAGE and np.all(codes[2] == 0) and dl[2] == 0.0
    assert st[3] & oracle.VERBATIM


def test_ae_exact_flag_when_all_codes_zero():
    x = synth.histograms(2, synth.config_seed(0))
    xh = np.zeros((2, 1536), np.float32)
    xh[:, :synth.P] = x.astype(np.float32)  # within Delta/2 everywhere
    codes, xp, scale, dl, st = oracle.quantize(x, xh, 1e-3)
    assert np.all(codes == 0)
    assert np.all(st & oracle.AE_EXACT)


def test_dequantize_reproduces_xprime():
    x = synth.histograms(6, synth.config_seed(0))
    xh = synth.stand_in_xhat(x, 8)
    xh[1, 3] = np.nan
    codes, xp, scale, dl, st = oracle.quantize(x, xh, 1e-4)
    back = oracle.dequantize(xh, codes, x, dl)
    assert np.array_equal(back, xp)


def test_zero_level_rule_edges():
    dl = 2.0 ** -14
    # x = 0: any positive or negative grid level loses to the zero level
    for xh in (1e-6, -1e-6, 3e-5, -3e-5):
        x = 0.0
        c = oracle.quantize(np.array([[x, 1.0]]), np.array([[xh, 1.0]], np.float32),
                            1e-4)[0][0, 0]
        assert c == exact_code(x, xh, dl)[0] == oracle.ZERO_CODE
    # exact tie |x - g| == x (g == 2x) keeps the grid level
    x = 3 * 2.0 ** -20
    xh = np.float32(6 * 2.0 ** -20)
    codes, xp, *_ = oracle.quantize(np.array([[x, 1.0]]), np.array([[xh, 1.0]], np.float32),
                                    1e-4)
    assert codes[0, 0] == 0 and xp[0, 0] == float(xh)
    assert exact_code(x, float(xh), dl) == (0, float(xh))
    # g = Delta - tiny rounds to Delta: grid level (distance Delta/2 - tiny) wins
    x = dl / 2
    codes, xp, *_ = oracle.quantize(np.array([[x, 1.0]]),
                                    np.array([[-1e-30, 1.0]], np.float32), 1e-4)
    assert codes[0, 0] == 1 and xp[0, 0] == dl
    assert exact_code(x, -1e-30, dl) == (1, dl)


def test_codes_random_vs_fraction_with_zero_level():
    rng = np.random.default_rng(21)
    n = 6
    x = synth.histograms(n, synth.config_seed(0))
    # decoded stand-in with strong absolute noise: many cells compete with 0
    xh = synth.stand_in_xhat(x, 22, rel=0.0, floor=3e-4)
    codes, xp, scale, dl, st = oracle.quantize(x, xh, 1e-3)
    nz = 0
    for b in range(n):
        for p in range(synth.P):
            ce, ve = exact_code(x[b, p], xh[b, p], dl[b])
            assert codes[b, p] == ce and xp[b, p] == ve
            nz += ce == oracle.ZERO_CODE
    assert nz > 100
