"""The paper's network shape (Sec. IV-B, Fig. 2): 33 x 37 histograms (37
v_par x 33 v_perp cells, P = 1221) and one tied linear layer with a latent of
4, through the whole path.

The one-layer model is the two-layer net with W2 = I and b2 = b3 = 0 held
fixed, so the FP64 oracle's network with those weights is its exact
reference: encoder/decoder outputs, the loss and the W1, b1, b4 gradients are
compared with it; the fixed layer stays the identity through training; the
compression of the 37 x 33 grid keeps both bounds and its codes equal the
oracle's quantizer on the GPU's decoded rows."""
import numpy as np
import pytest

import oracle
from paper_2212_10733_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"
GRID = (37, 33)
P, L = GRID[0] * GRID[1], 4


@pytest.fixture(scope="module")
def aq():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2212_10733_gb300 import aeqc
    aeqc.load()
    return aeqc


def params(seed):
    d = synth.ae_init(P, L, L, seed)
    rng = np.random.default_rng(seed)
    d["b1"] = rng.normal(0, 0.1, L)
    d["b4"] = rng.normal(0, 0.1, P)
    d["mu"] = rng.uniform(0, 0.3, P)
    d["sigma"] = rng.uniform(0.5, 1.5, P)
    return d


def oracle_net(d):
    # the one-layer net as the oracle's two-layer net with an identity layer
    return oracle.AE(W1=d["W1"], b1=d["b1"], W2=np.eye(L), b2=np.zeros(L), b3=np.zeros(L),
                     b4=d["b4"], mu=d["mu"], sigma=d["sigma"])


def test_shape_checks(aq):
    with pytest.raises(aq.AeqcError):
        aq.Model(P, 8, 4, layers=1)            # H must equal L
    with pytest.raises(aq.AeqcError):
        aq.Model(P, 4, 4, layers=1, tied=False)
    with pytest.raises(aq.AeqcError):
        aq.Model(P, 4, 4, layers=1, dtype=aq.DTYPE_BF16)


def test_forward_and_gradients_match_oracle(aq):
    d = params(3)
    m = aq.Model(P, L, L, layers=1)
    m.set_group(0, d)
    x = synth.histograms(200, synth.config_seed(6), grid=GRID)
    z, s = aq.ae_encode(m, torch.as_tensor(x, device=DEV))
    xh = aq.ae_decode(m, z, s)
    torch.cuda.synchronize()
    zo, xo, so = oracle.ae_forward(oracle_net(d), x)
    z, xh = z.cpu().numpy(), xh.cpu().numpy()[:, :P]
    assert np.all(np.abs(z - zo) <= 2e-4 * (np.abs(zo).max(axis=1, keepdims=True) + 1e-30))
    assert np.all(np.abs(xh - xo) <= 2e-4 * so[:, None])
    loss, g = m.loss_grad(torch.as_tensor(x[:32], device=DEV))
    lo, go = oracle.ae_loss_grad(oracle_net(d), x[:32])
    assert abs(loss.item() - lo) <= 1e-4 * lo
    g = g.cpu().numpy().astype(np.float64)
    o = 0
    for k, size in (("W1", P * L), ("b1", L), ("W2", L * L), ("b2", L), ("b3", L), ("b4", P)):
        got = g[o:o + size]
        o += size
        if k in ("W2", "b2", "b3"):
            assert np.all(got == 0.0), k  # the fixed layer does not train
        else:
            ref = go[k].ravel()
            assert np.all(np.abs(got - ref) <= 1e-3 * np.abs(ref).max() + 1e-12), k


def test_training_keeps_the_identity_and_compression_keeps_the_bounds(aq):
    xd = torch.as_tensor(synth.histograms(4096, synth.config_seed(6) + 1, grid=GRID),
                         device=DEV)
    m = aq.Model(P, L, L, layers=1)
    m.set_group(0, synth.ae_init(P, L, L, 9))
    m.fit_normalizer(0, xd[:1024])
    loss = torch.zeros(1, device=DEV)
    ws = None
    first = None
    for t in range(200):
        b = (t * 64) % 4000
        ws = m.train_step(xd[b:b + 64], lr=2e-3, loss_out=loss, ws=ws)
        if t == 0:
            first = loss.item()
    assert loss.item() < 0.7 * first
    gg = m.get_group(0)
    assert np.array_equal(gg["W2"], np.eye(L))
    assert not gg["b2"].any() and not gg["b3"].any()
    vpar, vperp, vol = synth.grid_arrays(*GRID)
    grid = aq.Grid(vpar, vperp, vol)
    og = oracle.Grid(vpar=vpar, vperp=vperp, vol_uniform=vol)
    p = aq.params_default(tau=1e-4, kernel=aq.KERNEL_FAST)
    comp = aq.compress_batch(m, grid, xd, p, outlier_capacity=xd.numel())
    f = aq.decompress_batch(m, grid, comp, p)
    xh = aq.ae_decode(m, comp.latent, comp.scale)
    torch.cuda.synchronize()
    x, f = xd.cpu().numpy(), f.cpu().numpy()
    st = comp.status.cpu().numpy()
    assert np.mean((st & aq.ST_VERBATIM) != 0) < 0.01
    assert np.all(np.abs(f - x) <= 1e-4 * x.max(axis=1, keepdims=True))
    S = oracle.abs_moments(og, x)
    assert np.all(np.abs(oracle.moments(og, f) - oracle.moments(og, x)) <= 1e-10 * S)
    # codes against the oracle's quantizer on the decoded rows (first level)
    rows = [r for r in range(0, 4096, 97) if not (st[r] & (aq.ST_ALPHA_RETRY | aq.ST_VERBATIM))]
    oc = oracle.quantize(x[rows], xh.cpu().numpy()[rows, :P], 1e-4)[0]
    np.testing.assert_array_equal(comp.codes.cpu().numpy()[rows], oc)
