"""Pins for the oracle's fallback paths and its decompression, against facts
that do not come from the oracle's own code.

* Round 2 (Sec. IV-E, the parameter study: a second Newton round with a
  smaller step, then verbatim storage), read as damped Newton from zero with
  backtracking on the dual.  Its success path is pinned by the closed form of
  the exponential tilt: x' = x exp(+lambda*.phi) has the unique solution
  lambda* (strict convexity), so a round that converges must return it.
  Round 1 is made to fail in two ways: an iteration cap of one step, and
  tilts so large that the undamped step of Eq. (6) overflows, which only a
  working line search survives.
* The alpha/4 retry of the end-to-end check: a decoded histogram biased by
  0.49 Delta leaves every residual at +0.49 Delta, so the correction at the
  alpha level moves the peak by several Delta and breaks the pointwise
  bound; at alpha/4 the same histogram quantizes to q = 2 with residuals of
  -0.04 Delta/4.  The retry's codes are checked against exact rational
  arithmetic at the alpha/4 bin width.
* Decompression (Sec. III, end of Stage 5): f = x' exp(-lambda.phi) with
  x' = xhat + q Delta (0 at the zero code, the raw value at escapes),
  recomputed here point by point with Python's own arithmetic on rows with
  the alpha/4 bin width, zero-level codes, escapes, verbatim storage and a
  zero image.
* Product quantisation of latents with non-finite values: such values take
  no part in training (the table equals the one trained without them) and
  encode as index 0.
"""
import math
from fractions import Fraction

import numpy as np

import oracle
from oracle import pq
from paper_2212_10733_gb300 import synth


def phi_matrix(grid):
    vp = np.tile(grid.vpar, len(grid.vperp))
    w = np.repeat(np.asarray(grid.vperp) ** 2, len(grid.vpar))
    return np.stack([np.ones_like(vp), vp, w, vp * vp])


def exact_delta(e: float, alpha: float) -> Fraction:
    """2^k with 2^k <= 2 alpha e < 2^(k+1), by exact comparisons."""
    budget = Fraction(2) * Fraction(alpha) * Fraction(e)
    k = 0
    while Fraction(2) ** k > budget:
        k -= 1
    while Fraction(2) ** (k + 1) <= budget:
        k += 1
    return Fraction(2) ** k


def exact_code(x: float, xh: float, dl: Fraction):
    """The quantizer's definition in rational arithmetic: q the round-half-even
    index of the exact (x - xhat) / Delta, escape beyond |q| = 32766 or for a
    non-finite xhat, the zero level when 0 is strictly nearer to x."""
    if not np.isfinite(xh):
        return oracle.ESCAPE
    q = round((Fraction(x) - Fraction(float(xh))) / dl)
    if abs(q) > oracle.CODE_MAX:
        return oracle.ESCAPE
    g = Fraction(float(xh)) + q * dl
    if Fraction(x) < abs(Fraction(x) - g):
        return oracle.ZERO_CODE
    return q


def tilted(grid, x, lam_true):
    return x * np.exp(lam_true @ phi_matrix(grid))


# --- round 2 -----------------------------------------------------------------

def test_round2_recovers_the_tilt_after_a_capped_round1(grid):
    x = synth.histograms(8, synth.config_seed(0))
    Q = oracle.moments(grid, x)
    rng = np.random.default_rng(21)
    lam_true = rng.normal(0, 1, size=(8, 4)) * np.array([3e-2, 1e-2, 3e-3, 3e-3])
    xp = tilted(grid, x, lam_true)
    pr = oracle.Params(max_iter=1)
    # one undamped step cannot reach 1e-12 from these tilts
    _, _, conv = oracle.newton_round1(grid, xp, Q, pr)
    assert not conv.any()
    lam, f, it, st = oracle.newton(grid, xp, Q, pr)
    assert np.all(st == oracle.ROUND2), st
    assert np.all(it > 1)
    np.testing.assert_allclose(lam, lam_true, rtol=0, atol=2e-11)
    np.testing.assert_allclose(f, x, rtol=1e-10, atol=1e-14 * x.max())


def test_round2_line_search_survives_overshooting_steps(grid):
    """Tilts of order one: the undamped step overflows or does not settle in
    50 steps; the damped round must still return the closed-form tilt."""
    x = synth.histograms(8, synth.config_seed(0))
    Q = oracle.moments(grid, x)
    rescued = 0
    for scale in (1.0, 2.0, 3.0, 5.0, 8.0):
        rng = np.random.default_rng(5)
        lam_true = rng.normal(0, 1, size=(8, 4)) * np.array([1.0, 0.5, 0.3, 0.2]) * scale
        xp = tilted(grid, x, lam_true)
        _, _, conv1 = oracle.newton_round1(grid, xp, Q, oracle.Params())
        lam, f, it, st = oracle.newton(grid, xp, Q, oracle.Params())
        fail1 = conv1 == 0
        # every histogram is solved: by round 1, or else by round 2
        assert np.all(st[~fail1] == oracle.CONVERGED)
        assert np.all(st[fail1] == oracle.ROUND2), (scale, st)
        assert np.all(np.abs(lam - lam_true) <= 5e-12 * (1 + np.abs(lam_true))), scale
        rescued += int(fail1.sum())
    assert rescued >= 15  # most of these tilts defeat the undamped step


def test_round2_inside_compress_correct(grid):
    """compress_correct hands a histogram that round 1 cannot solve within its
    cap to round 2: status ROUND2 (not CONVERGED), both bounds kept."""
    x = synth.histograms(16, synth.config_seed(0))
    xh = synth.stand_in_xhat(x, 41)
    pr = oracle.Params(tau=1e-4, max_iter=1)
    out = oracle.compress_correct(grid, x, xh, pr)
    st = out["status"]
    r2 = (st & oracle.ROUND2) != 0
    assert r2.sum() >= 8
    assert np.all((st[r2] & (oracle.CONVERGED | oracle.VERBATIM)) == 0)
    e = pr.tau * x.max(axis=1, keepdims=True)
    assert np.all(np.abs(out["f"] - x) <= e)
    Q, Qf, S = oracle.moments(grid, x), oracle.moments(grid, out["f"]), oracle.abs_moments(grid, x)
    assert np.all(np.abs(Qf - Q) / S <= 1e-11)
    # the same histograms with the default cap converge in round 1 to the same
    # multipliers (the solution is unique)
    ref = oracle.compress_correct(grid, x, xh, oracle.Params(tau=1e-4))
    same = (ref["status"] & oracle.ALPHA_RETRY) == (st & oracle.ALPHA_RETRY)
    M_ok = np.abs(ref["lam"][same] - out["lam"][same]).max()
    assert M_ok < 1e-9


# --- the alpha / 4 retry -------------------------------------------------------

def biased_batch(n=6, tau=1e-4, bias=0.49, seed=3):
    x = synth.histograms(n, synth.config_seed(0) + seed)
    s = x.max(axis=1)
    dl = np.array([float(exact_delta(tau * si, 0.5)) for si in s])
    xh = np.zeros((n, 1536), np.float32)
    xh[:, :x.shape[1]] = (x - bias * dl[:, None]).astype(np.float32)
    return x, xh, s


def test_alpha_retry_codes_are_the_exact_quantizer_at_alpha_over_4(grid):
    tau = 1e-4
    x, xh, s = biased_batch(tau=tau)
    pr = oracle.Params(tau=tau)
    out = oracle.compress_correct(grid, x, xh, pr)
    st = out["status"]
    retry = (st & oracle.ALPHA_RETRY) != 0
    assert retry.sum() >= 4
    assert np.all(st[retry] & oracle.CONVERGED)
    assert np.all((st & oracle.VERBATIM) == 0)
    P = x.shape[1]
    for b in np.nonzero(retry)[0]:
        dl4 = exact_delta(tau * s[b], 0.125)
        want = np.array([exact_code(float(x[b, p]), xh[b, p], dl4) for p in range(P)])
        np.testing.assert_array_equal(out["codes"][b], want)
        # mostly q = 2: (x - xhat) / (Delta / 4) = 1.96
        assert np.mean(want == 2) > 0.7
    e = tau * s[:, None]
    assert np.all(np.abs(out["f"] - x) <= e)
    Q, Qf, S = oracle.moments(grid, x), oracle.moments(grid, out["f"]), oracle.abs_moments(grid, x)
    assert np.all(np.abs(Qf - Q) / S <= 1e-12)


def test_alpha_level_breaks_the_bound_on_the_biased_batch(grid):
    """Why the retry happens: at the alpha level every residual is +0.49 Delta
    and the corrected peak moves by more than e.  Checked on an independent
    evaluation of f = x' exp(-lambda.phi) in numpy."""
    tau = 1e-4
    x, xh, s = biased_batch(tau=tau)
    codes, xp, _, _, _ = oracle.quantize(x, xh, tau, 0.5)
    Q = oracle.moments(grid, x)
    lam, _, _, st = oracle.newton(grid, xp, Q, oracle.Params(tau=tau))
    assert np.all(st & oracle.CONVERGED)
    f = xp * np.exp(-(lam @ phi_matrix(grid)))
    worst = (np.abs(f - x) / (tau * s[:, None])).max(axis=1)
    out = oracle.compress_correct(grid, x, xh, oracle.Params(tau=tau))
    retry = (out["status"] & oracle.ALPHA_RETRY) != 0
    assert np.all(worst[retry] > 1.0)
    assert np.all(worst[~retry] <= 1.0)


# --- decompression -----------------------------------------------------------

def hand_decompress(grid, xh_row, codes, raw, scale, lam, status, pr):
    """f = x' exp(-lambda.phi), point by point in Python floats."""
    P = grid.P
    if status & oracle.ZERO_IMAGE:
        return np.zeros(P)
    if status & (oracle.VERBATIM | oracle.NONFINITE_INPUT):
        dl = 0.0
    else:
        a = pr.alpha * (0.25 if status & oracle.ALPHA_RETRY else 1.0)
        dl = float(exact_delta(pr.tau * scale, a))
    n_par = len(grid.vpar)
    f = np.zeros(P)
    for p in range(P):
        j, i = divmod(p, n_par)
        c = int(codes[p])
        if c == oracle.ESCAPE:
            xp = float(raw[p])
        elif c == oracle.ZERO_CODE:
            xp = 0.0
        else:
            xp = float(xh_row[p]) + c * dl  # c * dl is exact; one rounding
        v, w = float(grid.vpar[i]), float(grid.vperp[j]) ** 2
        lp = lam[0] * 1.0 + lam[1] * v + lam[2] * w + lam[3] * (v * v)
        f[p] = xp * math.exp(-lp)
    return f


def test_decompress_against_a_hand_computation(grid):
    tau = 1e-4
    x, xh, s = biased_batch(n=5, tau=tau, seed=7)
    # row 3: escapes (non-finite and far-off decoded values) next to normal
    # points; row 4: a zero image
    xh[3, 100] = np.nan
    xh[3, 200] = np.float32(x[3, 200] + 5e4 * float(exact_delta(tau * s[3], 0.5)))
    x[4] = 0.0
    xh[4, :] = 0.0
    pr = oracle.Params(tau=tau)
    out = oracle.compress_correct(grid, x, xh, pr)
    st = out["status"]
    assert (st & oracle.ALPHA_RETRY).any() and (st[4] & oracle.ZERO_IMAGE)
    assert out["codes"][3, 100] == oracle.ESCAPE and out["codes"][3, 200] == oracle.ESCAPE
    assert (out["codes"] == oracle.ZERO_CODE).any()
    f = oracle.decompress(grid, xh, out["codes"], x, out["scale"], out["lam"], st, pr)
    for b in range(x.shape[0]):
        want = hand_decompress(grid, xh[b], out["codes"][b], x[b], out["scale"][b],
                               out["lam"][b], int(st[b]), pr)
        # the two sides may call different exp implementations: a few ulp
        np.testing.assert_allclose(f[b], want, rtol=4e-16, atol=0)
    # a verbatim row decompresses to the raw input exactly
    v = oracle.compress_correct(grid, x[:1], np.zeros((1, 1536), np.float32),
                                oracle.Params(tau=10.0, max_iter=5, r2_max_iter=5))
    assert v["status"][0] & oracle.VERBATIM
    fv = oracle.decompress(grid, np.zeros((1, 1536), np.float32), v["codes"], x[:1],
                           v["scale"], v["lam"], v["status"], oracle.Params(tau=10.0))
    np.testing.assert_array_equal(fv, x[:1])


def test_decompress_alpha_retry_uses_the_quarter_bin(grid):
    """A plausible slip (decompressing a retried row with the alpha bin width)
    moves x' by (3/4) q Delta: the oracle's f must match only the alpha/4 one."""
    tau = 1e-4
    x, xh, s = biased_batch(tau=tau)
    pr = oracle.Params(tau=tau)
    out = oracle.compress_correct(grid, x, xh, pr)
    st = out["status"]
    b = int(np.nonzero(st & oracle.ALPHA_RETRY)[0][0])
    f = oracle.decompress(grid, xh, out["codes"], x, out["scale"], out["lam"], st, pr)[b]
    wrong = hand_decompress(grid, xh[b], out["codes"][b], x[b], out["scale"][b], out["lam"][b],
                            int(st[b]) & ~oracle.ALPHA_RETRY, pr)
    assert np.abs(f - wrong).max() > 0.5 * float(exact_delta(tau * s[b], 0.125))
    assert np.all(np.abs(f - x[b]) <= tau * s[b])


# --- product quantisation: non-finite latents ---------------------------------

def test_pq_nonfinite_latents_are_left_out_of_training_and_coded_zero():
    rng = np.random.default_rng(8)
    z = rng.standard_normal((400, 3)).astype(np.float32)
    bad = rng.choice(400, size=30, replace=False)
    zb = z.copy()
    zb[bad[:10], 1] = np.nan
    zb[bad[10:20], 1] = np.inf
    zb[bad[20:], 1] = -np.inf
    k, iters = 8, 6
    c = pq.train(zb, k, iters)
    keep = np.ones(400, bool)
    keep[bad] = False
    # column 1 trained on its finite values alone; columns 0 and 2 untouched
    c1 = pq.train(z[keep][:, 1:2], k, iters)
    np.testing.assert_array_equal(c[1], c1[0])
    np.testing.assert_array_equal(c[[0, 2]], pq.train(z[:, [0, 2]], k, iters))
    codes = pq.assign(zb, c)
    assert np.all(codes[bad, 1] == 0)
    # finite values keep their nearest centroid (brute force)
    for r in np.nonzero(keep)[0][:50]:
        d = np.abs(np.float32(zb[r, 1]) - c[1])
        assert codes[r, 1] == int(np.argmin(d))
    # an all-non-finite column keeps the zero table
    zn = np.full((5, 1), np.nan, np.float32)
    np.testing.assert_array_equal(pq.train(zn, 4, 3), np.zeros((1, 4), np.float32))
