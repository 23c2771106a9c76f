"""Training step of the BF16 model (Eq. (5), Adam, Sec. III Stage 2 and
Sec. IV-B) on the tensor cores, through the C ABI, against the FP64 oracle.

The forward layers and the gradient products run as tcgen05 GEMMs with
BF16-rounded operands and FP32 accumulation, so the bar is the BF16 one:
the loss within 1e-2 relative and every gradient array within 1e-2 of its
largest entry (operands carry 2^-9 relative rounding through four layers).
The shapes span several 128-row and 128-column tiles, a ragged K tail
(P = 1521 = 23 x 64 + 49) and batches that are not a multiple of 128.  With
ReLU the bar is 3e-2: a hidden pre-activation within BF16 rounding of zero
takes its mask from the rounded value, so the masks of a few units differ
from the FP64 ones and their gradient terms with them (the paper's network
is linear, where no such decision exists).
"""
import numpy as np
import pytest

import oracle
from paper_2212_10733_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def aq():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2212_10733_gb300 import aeqc
    aeqc.load()
    return aeqc


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def rand_params(P, H, L, tied, seed):
    d = synth.ae_init(P, H, L, seed, tied=tied)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3", "b4"):
        d[k] = rng.normal(0, 0.1, size=d[k].shape)
    d["mu"] = rng.uniform(0, 0.3, size=P)
    d["sigma"] = rng.uniform(0.5, 1.5, size=P)
    return d


@pytest.mark.parametrize("H,L,B,tied,act", [
    (128, 16, 200, True, 0),
    (256, 32, 128, False, 0),
    (128, 32, 77, True, 1),
])
def test_bf16_loss_grad_matches_oracle(aq, H, L, B, tied, act):
    P = 1521
    prm = rand_params(P, H, L, tied, 17)
    m = aq.Model(P, H, L, tied=tied, act=act, dtype=aq.DTYPE_BF16)
    m.set_group(0, prm)
    x = synth.histograms(B, synth.config_seed(2))
    loss, g = m.loss_grad(dev(x))
    torch.cuda.synchronize()
    assert m.device_status() == 0
    lo, go = oracle.ae_loss_grad(oracle.AE(act=act, **prm), x)
    assert abs(loss.item() - lo) <= 1e-2 * lo
    g = g.cpu().numpy().astype(np.float64)
    order = ["W1", "b1", "W2", "b2"] + ([] if tied else ["W3"]) + ["b3"] + \
            ([] if tied else ["W4"]) + ["b4"]
    o = 0
    for k in order:
        ref = go[k].ravel()
        got = g[o:o + ref.size]
        o += ref.size
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= (3e-2 if act else 1e-2), (k, err)
    assert o == g.size
    m.close()


def test_bf16_training_reduces_loss_like_fp32(aq):
    """Sixty Adam steps from the same start: the BF16 model's loss falls as
    the FP32 model's does (within 5 %), and no bounded wait ran out."""
    P, H, L = 1521, 128, 16
    x = dev(synth.histograms(256, synth.config_seed(3)))
    init = synth.ae_init(P, H, L, 5)
    losses = {}
    for dt in (aq.DTYPE_F32, aq.DTYPE_BF16):
        m = aq.Model(P, H, L, dtype=dt)
        m.set_group(0, init)
        m.fit_normalizer(0, x)
        loss = torch.zeros(1, device=DEV)
        ws = None
        first = None
        for t in range(60):
            ws = m.train_step(x[(t % 2) * 128:(t % 2) * 128 + 128], lr=1e-3, loss_out=loss, ws=ws)
            if t == 0:
                first = loss.item()
        losses[dt] = (first, loss.item())
        assert m.device_status() == 0
        m.close()
    f32, b16 = losses[aq.DTYPE_F32], losses[aq.DTYPE_BF16]
    assert b16[1] < 0.5 * b16[0]
    assert abs(b16[1] - f32[1]) <= 0.05 * f32[1]


def bf16(a):
    """float32 -> nearest BF16 (ties to even), as float64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def emulate_loss_grad(p, x, tied):
    """The BF16 training step's arithmetic (identity activation) in numpy:
    each product of BF16-rounded FP32 operands summed in FP64, rounded to
    FP32 with its epilogue, the elementwise steps in FP32."""
    f32 = np.float32
    P = x.shape[1]
    B = x.shape[0]
    W1, b1, W2, b2 = (f32(p[k]) for k in ("W1", "b1", "W2", "b2"))
    b3, b4 = f32(p["b3"]), f32(p["b4"])
    W3 = W2.T if tied else f32(p["W3"])
    W4 = W1.T if tied else f32(p["W4"])
    mu, sig = f32(p["mu"]), f32(p["sigma"])
    s = x.max(axis=1, keepdims=True)
    u = f32((x * (1.0 / s) - mu.astype(np.float64)) / sig.astype(np.float64))
    mm = lambda a, b: f32(bf16(a) @ bf16(b))
    h1 = f32(mm(u, W1) + b1)
    z = f32(mm(h1, W2) + b2)
    h3 = f32(mm(z, W3) + b3)
    y = f32(mm(h3, W4) + b4)
    d = f32(y - u)
    loss = float((d.astype(np.float64) ** 2).sum() / (B * P))
    dy = f32(f32(2.0 / (B * P)) * d)
    g = {"b4": dy.sum(axis=0, dtype=np.float64)}
    if tied:
        gW1 = mm(dy.T, h3)
        dh3 = mm(dy, W1)
    else:
        g["W4"] = mm(h3.T, dy)
        dh3 = mm(dy, W4.T)
    g["b3"] = dh3.sum(axis=0, dtype=np.float64)
    if tied:
        gW2 = mm(dh3.T, z)
        dz = mm(dh3, W2)
    else:
        g["W3"] = mm(z.T, dh3)
        dz = mm(dh3, W3.T)
    g["b2"] = dz.sum(axis=0, dtype=np.float64)
    g["W2"] = f32(mm(h1.T, dz) + gW2) if tied else mm(h1.T, dz)
    dh1 = mm(dz, W2.T)
    g["b1"] = dh1.sum(axis=0, dtype=np.float64)
    g["W1"] = f32(mm(u.T, dh1) + gW1) if tied else mm(u.T, dh1)
    return loss, g


@pytest.mark.parametrize("H,L,B,tied", [(128, 16, 200, True), (256, 32, 128, False)])
def test_bf16_loss_grad_matches_bf16_emulation(aq, H, L, B, tied):
    """Tight bar against the same BF16 arithmetic (the products that split
    their K range over several CTAs included): loss within 1e-4 relative,
    gradients within 2e-3 of each array's largest entry (FP32 summation order
    and the rare BF16 rounding it flips)."""
    P = 1521
    prm = rand_params(P, H, L, tied, 23)
    m = aq.Model(P, H, L, tied=tied, act=0, dtype=aq.DTYPE_BF16)
    m.set_group(0, prm)
    x = synth.histograms(B, synth.config_seed(5))
    loss, g = m.loss_grad(dev(x))
    torch.cuda.synchronize()
    assert m.device_status() == 0
    le, ge = emulate_loss_grad(prm, x, tied)
    assert abs(loss.item() - le) <= 1e-4 * le
    g = g.cpu().numpy().astype(np.float64)
    order = ["W1", "b1", "W2", "b2"] + ([] if tied else ["W3"]) + ["b3"] + \
            ([] if tied else ["W4"]) + ["b4"]
    o = 0
    for k in order:
        ref = np.asarray(ge[k], dtype=np.float64).ravel()
        got = g[o:o + ref.size]
        o += ref.size
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= 2e-3, (k, err)
    assert o == g.size
    m.close()
