"""GPU parity of the residual quantizer and the QoI correction (Stages 4-5)
against the FP64 oracle, through the C ABI.

Bars: codes, scales, statuses and x' bit-exact (integer / exact decisions
given the same decoded input); lambda within 1e-9 relative (+1e-11 absolute:
both sides stop at |g_k|/S_k <= 1e-12, which leaves lambda ~1e-13 from the
unique optimum); corrected moments within 1e-10 of the targets (relative to
S_k); every point within the pointwise bound.
"""
import numpy as np
import pytest

import oracle
from paper_2212_10733_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def aq():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2212_10733_gb300 import aeqc
    aeqc.load()
    return aeqc


@pytest.fixture(scope="module")
def grids(aq):
    vpar, vperp, vol = synth.grid_arrays()
    return aq.Grid(vpar, vperp, vol), oracle.Grid(vpar=vpar, vperp=vperp, vol_uniform=vol)


DEV = "cuda:0"


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def special_batch(n, seed, tau):
    """Seeded histograms with edge cases planted: decoded NaN/Inf/huge values,
    a negative input, a zero image, a NaN input, exact quantizer ties."""
    x = synth.histograms(n, synth.config_seed(0) + seed)
    xh = synth.stand_in_xhat(x, seed)
    xh[0, 10] = np.nan
    xh[0, 11] = np.inf
    xh[0, 12] = 1e30
    x[1, 5] = -1.0
    x[2, :] = 0.0
    x[3, 7] = np.nan
    # exact ties x - xhat = (m + 1/2) Delta: max(x) = 1 fixes Delta = 2^floor(log2(tau));
    # xhat is a float32 near 0.5 or below, so xhat + (m + 1/2) Delta is exact in FP64
    dl = 2.0 ** np.floor(np.log2(tau))
    for b in (4, 5):
        mx = x[b].max()
        x[b] /= mx
        if b == 4:  # row 5 keeps the unscaled xhat: hundreds of escape codes
            xh[b, :1521] = (xh[b, :1521] / mx).astype(np.float32)
        top = int(np.argmax(x[b]))
        for p in range(0, 1521, 13):
            m = (p % 23) - 11
            h = float(np.float32(x[b, p]))
            v = h + (m + 0.5) * dl
            if p == top or v < 0.0 or v >= 1.0:
                continue
            xh[b, p] = np.float32(h)
            x[b, p] = v
    return x, xh


@pytest.mark.parametrize("n,tau", [(203, 1e-4), (64, 1e-3), (1, 1e-4)])
def test_quantize_bit_exact(aq, n, tau):
    x, xh = special_batch(max(n, 8), 3, tau)
    x, xh = x[:n], xh[:n]
    p = aq.params_default(tau=tau)
    r = aq.residual_quantize(dev(x), dev(xh), p, outlier_capacity=4 * 1521, want_xrec=True)
    torch.cuda.synchronize()
    codes, xp, scale, dl, st = oracle.quantize(x, xh, tau)
    assert np.array_equal(r["codes"].cpu().numpy(), codes)
    assert np.array_equal(r["scale"].cpu().numpy(), scale)
    assert np.array_equal(r["status"].cpu().numpy(), st)
    g = r["xrec"].cpu().numpy()
    both_nan = np.isnan(g) & np.isnan(xp)
    assert np.array_equal(np.where(both_nan, 0, g), np.where(both_nan, 0, xp))
    cnt = int(r["count"].item())
    esc = np.flatnonzero(codes.ravel() == oracle.ESCAPE)
    assert cnt == len(esc)
    idx = r["index"][:cnt].cpu().numpy()
    val = r["value"][:cnt].cpu().numpy()
    order = np.argsort(idx)
    assert np.array_equal(idx[order], esc)
    xv = x.ravel()[esc]
    assert np.array_equal(np.nan_to_num(val[order], nan=-7.0), np.nan_to_num(xv, nan=-7.0))


def test_dequantize_bit_exact(aq):
    x, xh = special_batch(40, 5, 1e-4)
    p = aq.params_default(tau=1e-4)
    r = aq.residual_quantize(dev(x), dev(xh), p, outlier_capacity=4 * 1521, want_xrec=True)
    back = aq.residual_dequantize(dev(xh), r["codes"], r["scale"], r["status"], p,
                                  outliers=r["outliers"])
    torch.cuda.synchronize()
    codes, xp, scale, dl, st = oracle.quantize(x, xh, 1e-4)
    ref = oracle.dequantize(xh, codes, x, dl)
    b = back.cpu().numpy()
    zero = (st & oracle.ZERO_IMAGE) != 0
    assert np.array_equal(np.nan_to_num(b[~zero], nan=-7.0), np.nan_to_num(ref[~zero], nan=-7.0))
    assert np.all(b[zero] == 0.0)


def test_moments_match_oracle(aq, grids):
    g, og = grids
    x = synth.histograms(131, synth.config_seed(2))
    Q = aq.qoi_moments(g, dev(x)).cpu().numpy()
    Qo = oracle.moments(og, x)
    S = oracle.abs_moments(og, x)
    # different summation order: |error| <= P * eps * S_k = 1521 * 1.1e-16 * S_k
    assert np.all(np.abs(Q - Qo) <= 1.7e-13 * S)
    one = np.zeros((1, 1521))
    one[0, 5 * 39 + 17] = 1.0
    Q1 = aq.qoi_moments(g, dev(one)).cpu().numpy()
    # same cell, same phi: equal up to the association of vol * v * v
    assert np.allclose(Q1, oracle.moments(og, one), rtol=4.5e-16, atol=0)


def lam_close(a, b):
    return np.all(np.abs(a - b) <= 1e-9 * np.abs(b) + 1e-11)


def phi_of(og):
    vp = np.tile(og.vpar, len(og.vperp))
    vq = np.repeat(og.vperp, len(og.vpar)) ** 2
    return np.stack([np.ones_like(vp), vp, vq, vp * vp])


def lam_metric_close(a, b, xp, og, slack=3e-12):
    """lambda is unique, but a solver stopping at |g_k| <= tol S_k only fixes it
    to within tol in the metric of M = sum vol phi phi^T x': two correct
    solvers on different paths differ by |M (a - b)|_k <= 2 tol S_k.  Rows
    with some S_k = 0 (nothing to correct in that moment) are left out
    explicitly; every compared multiplier must be finite."""
    phi = phi_of(og)
    worst, wrow = 0.0, -1
    for r in range(len(a)):
        M = og.vol_uniform * (phi * xp[r]) @ phi.T
        S = og.vol_uniform * (np.abs(phi) * xp[r]).sum(1)
        if not np.all(S > 0):
            continue
        assert np.all(np.isfinite(a[r])) and np.all(np.isfinite(b[r])), (r, a[r], b[r])
        e = np.max(np.abs(M @ (a[r] - b[r])) / S)
        assert np.isfinite(e), r
        if e > worst:
            worst, wrow = e, r
    if worst > slack:
        print("lambda metric: worst %.3e at row %d: %s vs %s" % (worst, wrow, a[wrow], b[wrow]))
    return worst <= slack


def level_check_value(og, x, xh, tau, alpha):
    """max |f - x| / e of the oracle at one quantizer level (FP64), for a
    single finite histogram: the value the end-to-end check compares with 1."""
    codes, xp, _, _, st = oracle.quantize(x[None], xh[None], tau, alpha)
    Q = oracle.moments(og, x[None])
    lam, f, it, nst = oracle.newton(og, xp, Q)
    return float(np.max(np.abs(f[0] - x) / (tau * x.max())))


def expected_codes(og, x, xh, tau, st_gpu, ref):
    """Codes every row must carry: the oracle's where the statuses agree; where
    they differ, the oracle's quantizer at the level the GPU chose (all escape
    codes for a verbatim row).  A status may differ only through the end-to-end
    check's decision at a level whose check value is on the bound (within
    1e-6): the two sides evaluate f in different arithmetic."""
    want = ref["codes"].copy()
    diff = np.nonzero(st_gpu != ref["status"])[0]
    for r in diff:
        flip = int(st_gpu[r]) ^ int(ref["status"][r])
        assert flip & (oracle.ALPHA_RETRY | oracle.VERBATIM), (r, st_gpu[r], ref["status"][r])
        lvl = 0.125 if (flip & oracle.ALPHA_RETRY) == 0 else 0.5
        v = level_check_value(og, x[r], xh[r], tau, lvl)
        assert abs(v - 1.0) <= 1e-6, (r, v, st_gpu[r], ref["status"][r])
        if st_gpu[r] & oracle.VERBATIM:
            want[r] = oracle.ESCAPE
        else:
            a = 0.125 if st_gpu[r] & oracle.ALPHA_RETRY else 0.5
            want[r] = oracle.quantize(x[r][None], xh[r][None], tau, a)[0][0]
    return want, diff


def xprime_at_level(x, xh, tau, status):
    """x' of the quantizer level each histogram ended at (alpha or alpha/4)."""
    xp = oracle.quantize(x, xh, tau, 0.5)[1]
    retry = (status & oracle.ALPHA_RETRY) != 0
    if retry.any():
        xp[retry] = oracle.quantize(x[retry], xh[retry], tau, 0.125)[1]
    return xp


def test_newton_matches_oracle_and_closed_forms(aq, grids):
    g, og = grids
    n = 97
    x = synth.histograms(n, synth.config_seed(3))
    xh = synth.stand_in_xhat(x, 9)
    codes, xp, scale, dl, st = oracle.quantize(x, xh, 1e-4)
    Q = oracle.moments(og, x)
    p = aq.params_default()
    r = aq.qoi_correct(g, dev(xp), dev(Q), p, want_f=True)
    torch.cuda.synchronize()
    lam_o, f_o, it_o, st_o = oracle.newton(og, xp, Q)
    assert np.array_equal(r["status"].cpu().numpy(), st_o)
    assert lam_close(r["lam"].cpu().numpy(), lam_o)
    assert np.all(np.abs(r["iters"].cpu().numpy().astype(int) - it_o) <= 1)
    f = r["f"].cpu().numpy()
    S = oracle.abs_moments(og, x)
    assert np.all(np.abs(oracle.moments(og, f) - Q) <= 1e-11 * S)
    # exponential tilt: x' = x exp(+lambda*.phi) is undone by lambda*
    vp = np.tile(og.vpar, 39)
    vq = np.repeat(og.vperp, 39)
    phi = np.stack([np.ones_like(vp), vp, vq * vq, vp * vp])
    rng = np.random.default_rng(1)
    lam_t = rng.normal(0, 1, size=(n, 4)) * np.array([3e-2, 1e-2, 3e-3, 3e-3])
    r = aq.qoi_correct(g, dev(x * np.exp(lam_t @ phi)), dev(Q), p)
    assert np.allclose(r["lam"].cpu().numpy(), lam_t, rtol=1e-9, atol=1e-12)
    # identity: no step, lambda exactly 0
    r = aq.qoi_correct(g, dev(x), dev(Q), p)
    assert np.all(r["lam"].cpu().numpy() == 0.0) and np.all(r["iters"].cpu().numpy() == 0)


def test_l2_variant_matches_oracle(aq, grids):
    g, og = grids
    x = synth.histograms(9, synth.config_seed(4))
    xp = x + 1e-3 * x.max() * np.random.default_rng(2).standard_normal(x.shape)
    Q = oracle.moments(og, x)
    p = aq.params_default(loss=1)
    r = aq.qoi_correct(g, dev(xp), dev(Q), p)
    lam_o, *_ = oracle.newton(og, xp, Q, oracle.Params(loss=1))
    assert lam_close(r["lam"].cpu().numpy(), lam_o)


def check_batch(aq, og, x, xh, tau, kernel, n_expect_conv=0.95, prm=None, oprm=None):
    """quantize_correct against oracle.compress_correct on every row: codes
    bit-exact (at the level each side chose), scales exact, statuses equal
    except end-to-end-check flips proven to sit on the bound, multipliers in
    the M-metric, every point within the bound, moments within 1e-10."""
    p = prm or aq.params_default(tau=tau, kernel=kernel)
    out = aq.quantize_correct(aq_grid(aq), dev(x), dev(xh), p, outlier_capacity=64 * 1521,
                              want_f=True)
    torch.cuda.synchronize()
    ref = oracle.compress_correct(og, x, xh, oprm or oracle.Params(tau=tau))
    st = out.status.cpu().numpy()
    want, diff = expected_codes(og, x, xh, tau, st, ref)
    assert len(diff) <= max(2, len(x) // 1000), (len(diff), st[diff], ref["status"][diff])
    codes = out.codes.cpu().numpy()
    bad = np.nonzero((codes != want).any(axis=1))[0]
    assert len(bad) == 0, (bad[:8], st[bad[:8]], ref["status"][bad[:8]])
    assert np.array_equal(out.scale.cpu().numpy(), ref["scale"])
    same = st == ref["status"]
    lam = out.lam.cpu().numpy()
    if kernel == aq.KERNEL_FP64:  # same iteration as the oracle: lambda agrees closely
        assert lam_close(lam[same], ref["lam"][same])
    fin_rows = same & np.isfinite(x).all(axis=1) & ((st & oracle.VERBATIM) == 0)
    xp = xprime_at_level(np.nan_to_num(x[fin_rows]), xh[fin_rows], tau,
                         ref["status"][fin_rows])
    assert lam_metric_close(lam[fin_rows], ref["lam"][fin_rows], xp, og)
    f = out.f.cpu().numpy()
    fin = np.isfinite(x).all(axis=1)
    e = tau * np.where(fin, np.nan_to_num(x).max(axis=1), 0)[:, None]
    assert np.all(np.abs(f[fin] - x[fin]) <= e[fin])
    good = fin & (x.min(axis=1) >= 0) & (x.max(axis=1) > 0)
    S = oracle.abs_moments(og, x[good])
    assert np.all(np.abs(oracle.moments(og, f[good]) - oracle.moments(og, x[good])) <= 1e-10 * S)
    assert np.mean((st & (oracle.CONVERGED | oracle.ROUND2)) != 0) >= n_expect_conv
    return out, ref


_GRID = {}


def aq_grid(aq):
    if "g" not in _GRID:
        vpar, vperp, vol = synth.grid_arrays()
        _GRID["g"] = aq.Grid(vpar, vperp, vol)
    return _GRID["g"]


@pytest.mark.parametrize("n,tau", [(256, 1e-4), (61, 1e-3)])
@pytest.mark.parametrize("kernel", ["fp64", "fast"])
def test_quantize_correct_matches_oracle(aq, grids, n, tau, kernel):
    _, og = grids
    x, xh = special_batch(n, 11, tau)
    k = aq.KERNEL_FP64 if kernel == "fp64" else aq.KERNEL_FAST
    check_batch(aq, og, x, xh, tau, k, n_expect_conv=0.9)


@pytest.mark.parametrize("kernel", ["fast", "fp64"])
def test_large_batch_matches_oracle(aq, grids, kernel):
    """9,001 histograms: beyond the correction kernel's resident warps (at most
    4 CTAs x 4 warps on each of the SMs), so warps take several histograms
    each and the last wave is ragged; every row against the oracle."""
    _, og = grids
    n = 9001
    x = synth.histograms(n, synth.config_seed(8))
    xh = synth.stand_in_xhat(x, 21)
    k = aq.KERNEL_FP64 if kernel == "fp64" else aq.KERNEL_FAST
    check_batch(aq, og, x, xh, 1e-4, k, n_expect_conv=0.99)


def test_round2_success_path_matches_oracle_tilts(aq, grids):
    """Tilts of order one defeat the undamped step of Eq. (6); round 2 (damped
    Newton from zero) must return the closed-form tilt, as the oracle does."""
    g, og = grids
    n = 48
    x = synth.histograms(n, synth.config_seed(0))
    Q = oracle.moments(og, x)
    rng = np.random.default_rng(5)
    lam_t = rng.normal(0, 1, size=(n, 4)) * np.array([1.0, 0.5, 0.3, 0.2]) * 2.0
    xp = x * np.exp(lam_t @ phi_of(og))
    r = aq.qoi_correct(g, dev(xp), dev(Q), aq.params_default())
    torch.cuda.synchronize()
    lam_o, f_o, it_o, st_o = oracle.newton(og, xp, Q)
    st = r["status"].cpu().numpy()
    assert np.array_equal(st, st_o)
    assert np.sum(st == oracle.ROUND2) >= 10
    lam = r["lam"].cpu().numpy()
    assert np.all(np.abs(lam - lam_t) <= 1e-11 * (1 + np.abs(lam_t)))
    assert lam_metric_close(lam, lam_o, xp, og)


@pytest.mark.parametrize("kernel", ["fast", "fp64"])
def test_round2_inside_quantize_correct_matches_oracle(aq, grids, kernel):
    """Round 1 capped at one step: most histograms go to round 2, in the FP64
    kernel (the fast kernel hands them over); codes, statuses and multipliers
    against the oracle with the same cap."""
    _, og = grids
    x, xh = special_batch(96, 17, 1e-4)
    k = aq.KERNEL_FP64 if kernel == "fp64" else aq.KERNEL_FAST
    p = aq.params_default(tau=1e-4, kernel=k, max_iter=1, warm_iters=1)
    out, ref = check_batch(aq, og, x, xh, 1e-4, k, n_expect_conv=0.9, prm=p,
                           oprm=oracle.Params(tau=1e-4, max_iter=1))
    st = out.status.cpu().numpy()
    assert np.sum((st & oracle.ROUND2) != 0) >= 48


def test_quantize_correct_verbatim_and_zero(aq, grids):
    _, og = grids
    x = synth.histograms(6, synth.config_seed(5))
    xh = np.zeros((6, 1536), np.float32)
    xh[:, 19] = 1.0  # decoder output supported on one column: infeasible for tau = 10
    p = aq.params_default(tau=10.0, max_iter=50, r2_max_iter=50)
    out = aq.quantize_correct(aq_grid(aq), dev(x), dev(xh), p, outlier_capacity=8 * 1521,
                              want_f=True)
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()
    assert np.all(st & oracle.VERBATIM)
    assert np.array_equal(out.f.cpu().numpy(), x)
    assert int(out.count.item()) == 6 * 1521
    ref = oracle.compress_correct(og, x, xh, oracle.Params(tau=10.0, max_iter=50,
                                                           r2_max_iter=50))
    assert np.array_equal(st, ref["status"])


def test_outlier_overflow_is_reported(aq):
    x, xh = special_batch(8, 7, 1e-4)
    p = aq.params_default(tau=1e-4)
    r = aq.residual_quantize(dev(x), dev(xh), p, outlier_capacity=2)
    torch.cuda.synchronize()
    st = r["status"].cpu().numpy()
    assert int(r["count"].item()) > 2
    assert np.any(st & aq.ST_OUTLIER_OVERFLOW)


def test_empty_batch_is_a_noop(aq, grids):
    g, _ = grids
    x = torch.empty((0, 1521), dtype=torch.float64, device=DEV)
    Q = aq.qoi_moments(g, x)
    assert Q.shape == (0, 4)


def biased_xhat(x, tau, pattern, og):
    """Decoded histograms that leave residuals of a chosen sign pattern
    (rho Delta, |rho| <= 0.45): large moment defects, so the multipliers reach
    the fast kernel's limits (|lambda.phi| up to 0.05, |H| up to 1e-5 S)."""
    v = np.tile(og.vpar, len(og.vperp)) / 4.0
    rho = {"cubic": 0.45 * v ** 3, "quad": 0.45 * (2 * v * v - 1),
           "const": 0.45 * np.ones_like(v)}[pattern]
    dl = np.array([oracle.delta(tau * s, 0.5) for s in x.max(axis=1)])
    xh = np.zeros((len(x), 1536), np.float32)
    xh[:, :x.shape[1]] = (x - rho[None, :] * dl[:, None]).astype(np.float32)
    return xh


@pytest.mark.parametrize("tau,pattern", [(1e-3, "cubic"), (3e-3, "cubic"), (3e-3, "quad"),
                                         (3e-3, "const"), (1e-2, "const")])
def test_fast_kernel_converged_means_residual_below_tol(aq, grids, tau, pattern):
    """Every histogram the fast kernel reports converged has |g_k| <= 1e-12 S_k
    (reading of the stopping rule: S_k = sum vol |phi_k| f at the final
    lambda), recomputed here in FP64 from its multipliers with exactly
    rounded sums (math.fsum): the kernel's truncated series for h(t), its FP32
    sums and its certified last step must all be inside the bound.  The
    inputs sit near the kernel's limits (checked: some rows reach
    |lambda.phi| > 0.02 and |H| > 3e-6 S)."""
    import math
    _, og = grids
    x = synth.histograms(64, synth.config_seed(0) + 50)
    xh = biased_xhat(x, tau, pattern, og)
    p = aq.params_default(tau=tau, kernel=aq.KERNEL_FAST)
    out = aq.quantize_correct(aq_grid(aq), dev(x), dev(xh), p, want_f=True)
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()
    lam = out.lam.cpu().numpy()
    codes = out.codes.cpu().numpy()
    phi = phi_of(og)
    vol = og.vol_uniform
    reach_t, reach_h = 0.0, 0.0
    for b in np.nonzero(st & oracle.CONVERGED)[0]:
        a = 0.125 if st[b] & oracle.ALPHA_RETRY else 0.5
        qc, xp, _, _, _ = oracle.quantize(x[b][None], xh[b][None], tau, a)
        assert np.array_equal(qc[0], codes[b]), b
        xp = xp[0]
        t = lam[b] @ phi
        f = xp * np.exp(-t)
        for k in range(4):
            gk = math.fsum(vol * phi[k] * (f - x[b]))
            Sk = math.fsum(vol * np.abs(phi[k]) * f)
            assert abs(gk) <= (1e-12 + 1e-15) * Sk, (b, k, abs(gk) / Sk)
        pos = xp > 0
        reach_t = max(reach_t, float(np.abs(t[pos]).max()))
        h = np.expm1(-t) + t
        Hs = np.abs(vol * (phi * xp * h).sum(1)) / (vol * (np.abs(phi) * xp).sum(1))
        if np.abs(t[pos]).max() <= 0.05 and Hs.max() <= 1e-5:
            reach_h = max(reach_h, float(Hs.max()))
    assert np.mean((st & oracle.CONVERGED) != 0) >= 0.9
    if (tau, pattern) == (3e-3, "quad"):
        assert reach_t > 0.02 and reach_h > 3e-6, (reach_t, reach_h)


@pytest.mark.parametrize("kernel", ["fast", "fp64"])
def test_verbatim_after_the_retry_matches_oracle(aq, grids, kernel):
    """Heavy-tailed histograms whose corrected output breaks the pointwise
    bound at alpha and again at alpha / 4 are stored verbatim (status
    VERBATIM | ALPHA_RETRY, every code an escape, f = x, lambda = 0): the fast
    kernel stores them itself when the violation is certain, as the oracle
    and the FP64 kernel do."""
    _, og = grids
    x = synth.histograms(400, synth.config_seed(0) + 61, k_max=4, heavy_frac=1.0)
    xh = synth.stand_in_xhat(x, 61)
    k = aq.KERNEL_FP64 if kernel == "fp64" else aq.KERNEL_FAST
    out, ref = check_batch(aq, og, x, xh, 1e-4, k, n_expect_conv=0.9)
    st = out.status.cpu().numpy()
    vb = st == (oracle.VERBATIM | oracle.ALPHA_RETRY)
    assert vb.sum() >= 5
    assert np.all(out.lam.cpu().numpy()[vb] == 0.0)
    assert np.array_equal(out.f.cpu().numpy()[vb], x[vb])
    assert np.all(out.codes.cpu().numpy()[vb] == oracle.ESCAPE)


def carry_maxima(tau, count):
    """Row maxima s at which fl(tau s) lands exactly on a power of two although
    tau s is below it (the rounding carries into the next binade: Delta doubles
    there), each paired with the largest s whose product stays below."""
    from fractions import Fraction
    import math
    carry, below = [], []
    for m in range(-10, 30):
        t = math.ldexp(1.0, m) / tau
        s = t
        for _ in range(8):
            if tau * s == math.ldexp(1.0, m) and Fraction(tau) * Fraction(s) < Fraction(2) ** m:
                carry.append(s)
            elif tau * s < math.ldexp(1.0, m):
                below.append(s)
                break
            s = math.nextafter(s, 0.0)
        if len(carry) >= count:
            break
    return carry[:count], below[:count]


# (whether such maxima exist depends on tau's significand alone: for 1e-4
# they do not, for 1.1e-4 and 3e-3 at every power of two)
@pytest.mark.parametrize("tau", [1.1e-4, 3e-3])
def test_bin_width_at_binade_carries_matches_oracle(aq, grids, tau):
    """The fast kernel takes the bin width's exponent from the integer
    significand product of tau and max(x) (Sec. III Stage 4: Delta =
    2^floor(log2(2 alpha tau max x)) with the products rounded in float64).
    Rows whose maximum makes fl(tau s) round up onto a power of two, and rows
    just below such a boundary, must get the oracle's Delta, codes, scale and
    status."""
    _, og = grids
    carry, below = carry_maxima(tau, 16)
    assert len(carry) >= 8
    svals = np.array(carry + below)
    x = synth.histograms(len(svals), synth.config_seed(0) + 71)
    for r, s in enumerate(svals):
        k = int(np.argmax(x[r]))
        x[r] *= (s / x[r, k]) * (1.0 - 1e-9)
        x[r, k] = s
    assert np.array_equal(x.max(axis=1), svals)
    xh = synth.stand_in_xhat(x, 72)
    check_batch(aq, og, x, xh, tau, aq.KERNEL_FAST, n_expect_conv=0.9)
    dl = np.array([oracle.delta(tau * s, 0.5) for s in svals])
    assert len(np.unique(np.log2(dl[:len(carry)]))) > 1  # several binades
