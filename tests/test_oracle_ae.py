"""Pins for the oracle's autoencoder (Stage 2/3: dense layers, MSE loss of
Eq. (5), Adam), the warm-start MLP and NRMSE (Eq. (7)).

Independent references: numpy matrix products (library primitive), central
finite differences in FP64, the closed form of Adam's first step, textbook
NRMSE values and numpy mean/std.  The trajectory of trained weights over many
steps has no such pin (parity unpinned; only loss curves are compared).
"""
import numpy as np
import pytest

import oracle
from paper_2212_10733_gb300 import synth


def np_forward(d, x, act=0, tied=True):
    a = (lambda v: np.maximum(v, 0.0)) if act == 1 else (lambda v: v)
    s = x.max(axis=1, keepdims=True)
    u = (x / s - d["mu"]) / d["sigma"]
    h1 = a(u @ d["W1"] + d["b1"])
    z = h1 @ d["W2"] + d["b2"]
    W3 = d["W2"].T if tied else d["W3"]
    W4 = d["W1"].T if tied else d["W4"]
    h3 = a(z @ W3 + d["b3"])
    y = h3 @ W4 + d["b4"]
    return z, s * (d["sigma"] * y + d["mu"]), s[:, 0], u, y


def rand_ae(P, H, L, tied, seed, act=0):
    d = synth.ae_init(P, H, L, seed, tied=tied)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3", "b4"):
        d[k] = rng.normal(0, 0.1, size=d[k].shape)
    d["mu"] = rng.uniform(0, 0.5, size=P)
    d["sigma"] = rng.uniform(0.5, 1.5, size=P)
    return oracle.AE(act=act, **d), d


@pytest.mark.parametrize("tied", [True, False])
@pytest.mark.parametrize("act", [0, 1])
def test_forward_matches_numpy(tied, act):
    P, H, L = 1521, 16, 4
    m, d = rand_ae(P, H, L, tied, 3, act)
    x = synth.histograms(12, synth.config_seed(0))
    z, xh, s = oracle.ae_forward(m, x)
    z2, xh2, s2, _, _ = np_forward(d, x, act, tied)
    assert np.array_equal(s, s2)
    assert np.allclose(z, z2, rtol=1e-12, atol=1e-12)
    assert np.allclose(xh, xh2, rtol=1e-12, atol=1e-13)
    xd = oracle.ae_decode(m, z, s)
    assert np.allclose(xd, xh, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("tied", [True, False])
@pytest.mark.parametrize("act", [0, 1])
def test_gradient_matches_finite_differences(tied, act):
    P, H, L, B = 9, 4, 2, 3
    rng = np.random.default_rng(5)
    m, d = rand_ae(P, H, L, tied, 7, act)
    x = rng.uniform(0.1, 2.0, size=(B, P))
    loss, g = oracle.ae_loss_grad(m, x)
    _, _, _, u, y = np_forward(d, x, act, tied)
    assert abs(loss - np.mean((y - u) ** 2)) <= 1e-14 * max(1.0, loss)
    h = 1e-6
    for name, grad in g.items():
        arr = getattr(m, name)
        flat = arr.reshape(-1)
        for t in range(flat.size):
            old = flat[t]
            flat[t] = old + h
            lp, _ = oracle.ae_loss_grad(m, x)
            flat[t] = old - h
            lm, _ = oracle.ae_loss_grad(m, x)
            flat[t] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad.reshape(-1)[t]) <= 1e-7 * max(1.0, abs(fd)), (name, t)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(8)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    w0 = w.copy()
    m1, m2 = np.zeros(50), np.zeros(50)
    oracle.adam(w, g, m1, m2, lr=1e-3, t=1)
    # first step: m_hat = g, v_hat = g^2  =>  w -= lr g / (|g| + eps)
    assert np.allclose(w, w0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # second step with the same gradient keeps m_hat = g, v_hat = g^2
    w1 = w.copy()
    oracle.adam(w, g, m1, m2, lr=1e-3, t=2)
    assert np.allclose(w, w1 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)


def test_training_reduces_loss_on_synthetic_data():
    P, H, L = 1521, 16, 4
    x = synth.histograms(64, synth.config_seed(0))
    d = synth.ae_init(P, H, L, 11)
    mu, sd = oracle.fit_normalizer(x, P)
    d["mu"], d["sigma"] = mu, sd
    m = oracle.AE(**d)
    names = ("W1", "b1", "W2", "b2", "b3", "b4")
    mom = {k: (np.zeros_like(getattr(m, k)), np.zeros_like(getattr(m, k))) for k in names}
    losses = []
    for t in range(1, 31):
        loss, g = oracle.ae_loss_grad(m, x)
        losses.append(loss)
        for k in names:
            oracle.adam(getattr(m, k), g[k], *mom[k], lr=1e-3, t=t)
    assert losses[-1] < 0.5 * losses[0]


def test_fit_normalizer_matches_numpy():
    x = synth.histograms(40, synth.config_seed(0))
    mu, sd = oracle.fit_normalizer(x, synth.P, floor_sigma=1e-6)
    r = x / x.max(axis=1, keepdims=True)
    assert np.allclose(mu, r.mean(axis=0), rtol=1e-13, atol=1e-16)
    assert np.allclose(sd, np.maximum(r.std(axis=0), 1e-6), rtol=1e-10, atol=1e-16)


def test_mlp_forward_and_gradients():
    nin, nh, no, B = 6, 5, 4, 4
    rng = np.random.default_rng(12)
    d = synth.mlp_init(nin, nh, no, 3)
    for k in ("b1", "b2", "b3"):
        d[k] = rng.normal(0, 0.2, size=d[k].shape)
    m = oracle.MLP(in_mu=rng.normal(size=nin), in_sd=rng.uniform(0.5, 2, nin),
                   out_mu=rng.normal(size=no), out_sd=rng.uniform(0.5, 2, no), **d)
    inp = rng.normal(size=(B, nin))
    tgt = rng.normal(size=(B, no))
    u = (inp - m.in_mu) / m.in_sd
    h1 = np.maximum(u @ m.W1 + m.b1, 0)
    h2 = np.maximum(h1 @ m.W2 + m.b2, 0)
    o = h2 @ m.W3 + m.b3
    assert np.allclose(oracle.mlp_predict(m, inp), o * m.out_sd + m.out_mu, rtol=1e-13)
    loss, g = oracle.mlp_loss_grad(m, inp, tgt)
    t = (tgt - m.out_mu) / m.out_sd
    assert abs(loss - np.mean((o - t) ** 2)) < 1e-13
    h = 1e-6
    for name, grad in g.items():
        flat = getattr(m, name).reshape(-1)
        for k in range(flat.size):
            old = flat[k]
            flat[k] = old + h
            lp, _ = oracle.mlp_loss_grad(m, inp, tgt)
            flat[k] = old - h
            lm, _ = oracle.mlp_loss_grad(m, inp, tgt)
            flat[k] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad.reshape(-1)[k]) <= 1e-7 * max(1.0, abs(fd)), (name, k)


def test_nrmse_textbook_values():
    u = np.array([0.0, 1.0, 2.0, 3.0])
    assert oracle.nrmse(u, u) == 0.0
    assert abs(oracle.nrmse(u, u + 0.1) - 0.1 / 3.0) < 1e-15
    f = u.copy()
    f[2] += 0.4  # sqrt(0.16 / 4) / 3
    assert abs(oracle.nrmse(u, f) - 0.2 / 3.0) < 1e-15
