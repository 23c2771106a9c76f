"""Pins for the oracle's QoI moments (Eq. (1)-(4)) and the Newton correction
(Stage 5, Eq. (6)).

What fixes the answers here, independently of the oracle's own code:
  * one-hot histograms have moments vol * phi at that cell (index order, phi);
  * the four QoIs derived from the moments equal the direct integrals of
    Eq. (1)-(4) (algebraic identity, T_par with (v_par - u)^2 inside);
  * exact rational sums on a tiny grid;
  * x' = x needs no correction (lambda = 0, no step);
  * an exponential tilt x' = x exp(+lambda*.phi) is undone by lambda*;
  * a uniform scale x' = c x is undone by lambda = (log c, 0, 0, 0);
  * the first Newton step from 0 equals the x'-weighted least-squares
    projection, solved as a dense KKT system on tiny grids;
  * the L2-loss variant equals the unweighted KKT projection;
  * a 4x4 solve against numpy.linalg.solve.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2212_10733_gb300 import synth


def small_grid(n_par, n_perp, vol=None):
    vpar = np.linspace(-2.0, 3.0, n_par)
    vperp = np.linspace(0.25, 2.0, n_perp)
    return oracle.Grid(vpar=vpar, vperp=vperp, vol_uniform=0.37, vol=vol, mass=2.0)


def phi_matrix(g):
    """Phi [4][P] with P index = j * n_par + i."""
    vp = np.tile(g.vpar, len(g.vperp))
    vq = np.repeat(g.vperp, len(g.vpar))
    return np.stack([np.ones_like(vp), vp, vq * vq, vp * vp])


def vol_vector(g):
    if g.vol is not None:
        return g.vol.ravel()
    return np.full(g.P, g.vol_uniform)


def test_one_hot_moments_fix_index_order(grid):
    for (j, i) in [(0, 0), (0, 38), (38, 0), (5, 17), (20, 33)]:
        x = np.zeros(grid.P)
        x[j * 39 + i] = 1.0
        Q = oracle.moments(grid, x)[0]
        vp, vq = grid.vpar[i], grid.vperp[j]
        exp = grid.vol_uniform * np.array([1.0, vp, vq * vq, vp * vp])
        assert np.array_equal(Q, exp), (j, i, Q, exp)


def test_moments_exact_rational_tiny_grid():
    rng = np.random.default_rng(3)
    vol = rng.uniform(0.5, 1.5, size=(3, 4))
    g = small_grid(4, 3, vol=vol)
    x = rng.uniform(0, 10, size=(5, g.P))
    Q = oracle.moments(g, x)
    ph = phi_matrix(g)
    for b in range(5):
        for k in range(4):
            exact = sum(Fraction(vol.ravel()[p]) * Fraction(ph[k, p]) * Fraction(x[b, p])
                        for p in range(g.P))
            assert abs(Q[b, k] - float(exact)) <= 1e-14 * float(abs(exact)) + 1e-300


def test_derived_qois_equal_direct_integrals(grid):
    x = synth.histograms(32, synth.config_seed(0))
    Q = oracle.moments(grid, x)
    a = oracle.qois_from_moments(Q, mass=1.0)
    b = oracle.qois_direct(grid, x)
    assert np.allclose(a[:, 0], b[:, 0], rtol=1e-14, atol=0)
    assert np.allclose(a[:, 1], b[:, 1], rtol=1e-12, atol=1e-14)
    assert np.allclose(a[:, 2:], b[:, 2:], rtol=1e-12, atol=0)
    # non-unit mass scales the temperatures only
    g2 = oracle.Grid(vpar=grid.vpar, vperp=grid.vperp, vol_uniform=grid.vol_uniform, mass=3.5)
    c = oracle.qois_direct(g2, x)
    assert np.allclose(c[:, 2:], 3.5 * b[:, 2:], rtol=1e-14)


def test_moments_linear(grid):
    x = synth.histograms(4, synth.config_seed(0))
    y = synth.histograms(4, synth.config_seed(1))
    Qx, Qy = oracle.moments(grid, x), oracle.moments(grid, y)
    Qz = oracle.moments(grid, 2.0 * x + 0.5 * y)
    assert np.allclose(Qz, 2 * Qx + 0.5 * Qy, rtol=1e-13)


def test_identity_needs_no_correction(grid):
    x = synth.histograms(16, synth.config_seed(0))
    Q = oracle.moments(grid, x)
    lam, f, it, st = oracle.newton(grid, x, Q)
    assert np.array_equal(lam, np.zeros_like(lam))
    assert np.all(it == 0)
    assert np.all(st == oracle.CONVERGED)
    assert np.array_equal(f, x)


def test_exponential_tilt_is_undone(grid):
    x = synth.histograms(16, synth.config_seed(0))
    Q = oracle.moments(grid, x)
    ph = phi_matrix(grid)
    rng = np.random.default_rng(4)
    lam_true = rng.normal(0, 1, size=(16, 4)) * np.array([3e-2, 1e-2, 3e-3, 3e-3])
    xp = x * np.exp(lam_true @ ph)
    lam, f, it, st = oracle.newton(grid, xp, Q)
    assert np.all(st & oracle.CONVERGED)
    assert np.all(it <= 6)
    assert np.allclose(lam, lam_true, rtol=1e-9, atol=1e-12)
    assert np.allclose(f, x, rtol=1e-10, atol=1e-14 * x.max())


def test_uniform_scale_is_undone(grid):
    x = synth.histograms(8, synth.config_seed(0))
    Q = oracle.moments(grid, x)
    for c in (0.5, 1.001, 3.0):
        lam, f, it, st = oracle.newton(grid, c * x, Q)
        assert np.all(st & oracle.CONVERGED)
        # the stopping rule |g_k|/S_k <= 1e-12 leaves lambda off by ~1e-12 absolute
        assert np.allclose(lam[:, 0], np.log(c), rtol=0, atol=1e-11)
        assert np.allclose(lam[:, 1:], 0.0, atol=1e-11)


def kkt_solve(g, xp, Q, weights):
    """Dense KKT of min 1/2 sum (vol/weight)(f - x')^2 s.t. A f = Q with
    A = phi * vol; returns (f, mu).  weights = x' (KL linearisation) or 1 (L2)."""
    P = g.P
    A = phi_matrix(g) * vol_vector(g)[None, :]
    K = np.zeros((P + 4, P + 4))
    K[:P, :P] = np.diag(vol_vector(g) / weights)
    K[:P, P:] = A.T
    K[P:, :P] = A
    rhs = np.concatenate([vol_vector(g) / weights * xp, Q])
    sol = np.linalg.solve(K, rhs)
    return sol[:P], sol[P:]


@pytest.mark.parametrize("shape", [(3, 3), (4, 5), (5, 5)])
def test_first_newton_step_is_weighted_projection(shape):
    n_par, n_perp = shape
    rng = np.random.default_rng(n_par * 10 + n_perp)
    vol = rng.uniform(0.5, 1.5, size=(n_perp, n_par))
    g = small_grid(n_par, n_perp, vol=vol)
    for _ in range(5):
        x = rng.uniform(0.5, 2.0, size=g.P)
        xp = x * (1 + rng.normal(0, 0.05, size=g.P))
        Q = oracle.moments(g, x)[0]
        p1 = oracle.Params(max_iter=1, tol=0.0)
        lam, it, conv = oracle.newton_round1(g, xp, Q, p1)
        assert it[0] == 1
        f_lin, mu = kkt_solve(g, xp, Q, xp)
        assert np.allclose(lam[0], mu, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("shape", [(3, 3), (4, 5), (39, 39)])
def test_l2_variant_is_unweighted_projection(shape):
    n_par, n_perp = shape
    rng = np.random.default_rng(7)
    g = small_grid(n_par, n_perp)
    x = rng.uniform(0.5, 2.0, size=g.P)
    xp = x + rng.normal(0, 0.05, size=g.P)
    Q = oracle.moments(g, x)[0]
    pr = oracle.Params(loss=1)
    lam, f, it, st = oracle.newton(g, xp, Q, pr)
    f_kkt, mu = kkt_solve(g, xp, Q, np.ones(g.P))
    assert st[0] & oracle.CONVERGED
    assert it[0] <= 2
    assert np.allclose(lam[0], mu, rtol=1e-8, atol=1e-12)
    assert np.allclose(f[0], f_kkt, rtol=1e-10, atol=1e-12)


def test_cholesky_solve_vs_numpy():
    rng = np.random.default_rng(9)
    for _ in range(50):
        B = rng.normal(size=(4, 4))
        M = B @ B.T + 0.1 * np.eye(4)
        r = rng.normal(size=4)
        rc, d = oracle.cholesky_solve4(M, r)
        assert rc == 0
        assert np.allclose(d, np.linalg.solve(M, r), rtol=1e-10, atol=1e-12)
    rc, _ = oracle.cholesky_solve4(-np.eye(4), np.ones(4))
    assert rc == -1


def test_warm_start_from_the_solution_takes_no_step(grid):
    x = synth.histograms(8, synth.config_seed(0))
    xh = synth.stand_in_xhat(x, 11)
    pr = oracle.Params(tau=1e-4)
    codes, xp, scale, dl, st = oracle.quantize(x, xh, pr.tau)
    Q = oracle.moments(grid, x)
    lam, f, it, st = oracle.newton(grid, xp, Q, pr)
    lam_w, f_w, it_w, st_w = oracle.newton(grid, xp, Q, pr, lam0=lam)
    assert np.all(it_w == 0) and np.array_equal(lam_w, lam)
    # a poor warm start is rejected and the cold answer is recovered
    bad = lam + 1.0
    lam_b, f_b, it_b, st_b = oracle.newton(grid, xp, Q, pr, lam0=bad)
    assert np.all(st_b & oracle.WARM_REJECTED)
    assert np.allclose(lam_b, lam, rtol=1e-9, atol=1e-13)


def test_compress_correct_on_synthetic_batch(grid):
    n = 48
    x = synth.histograms(n, synth.config_seed(0))
    xh = synth.stand_in_xhat(x, 12)
    pr = oracle.Params(tau=1e-4)
    out = oracle.compress_correct(grid, x, xh, pr)
    st = out["status"]
    assert np.all(st & oracle.CONVERGED)
    assert np.all((st & oracle.VERBATIM) == 0)
    f = out["f"]
    e = pr.tau * x.max(axis=1, keepdims=True)
    assert np.all(np.abs(f - x) <= e)
    Q, Qf, S = oracle.moments(grid, x), oracle.moments(grid, f), oracle.abs_moments(grid, x)
    assert np.all(np.abs(Qf - Q) / S <= 1e-12)
    # decompression from codes + lambda reproduces f
    f2 = oracle.decompress(grid, xh, out["codes"], x, out["scale"], out["lam"], st, pr)
    assert np.array_equal(f2, f)
    # the round-1 convergence rate the paper reports (>= 99.5% at s = 1, 50 it)
    assert np.mean(out["iters"] <= 50) >= 0.995


def test_infeasible_target_goes_verbatim(grid):
    x = synth.histograms(2, synth.config_seed(0))
    xh = np.zeros((2, 1536), np.float32)
    # decoded histogram supported on one column only: the quantizer keeps the
    # bound, but a huge tau makes every code zero and x' cannot match 4 moments
    xh[:, :synth.P] = 0.0
    xh[:, 19] = 1.0
    pr = oracle.Params(tau=10.0, max_iter=50, r2_max_iter=50)
    out = oracle.compress_correct(grid, x, xh, pr)
    assert np.all(out["status"] & oracle.VERBATIM)
    assert np.array_equal(out["f"], x)
    assert np.all(out["codes"] == oracle.ESCAPE)
    assert np.all(out["lam"] == 0.0)


def test_zero_and_nonfinite_images(grid):
    x = synth.histograms(3, synth.config_seed(0))
    x[0] = 0.0
    x[1, 100] = np.inf
    xh = synth.stand_in_xhat(np.nan_to_num(x, posinf=1.0), 13)
    out = oracle.compress_correct(grid, x, xh, oracle.Params())
    assert out["status"][0] & oracle.ZERO_IMAGE and np.all(out["f"][0] == 0.0)
    assert out["status"][1] & oracle.VERBATIM
    assert np.array_equal(out["f"][1], x[1])
    assert out["status"][2] & oracle.CONVERGED
