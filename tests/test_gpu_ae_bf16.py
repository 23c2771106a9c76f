"""BF16 autoencoder forward on the tensor cores (tcgen05) through the C ABI.

Two references.  (1) A numpy restatement of the same arithmetic: inputs and
weights rounded to BF16 exactly as the kernels round them, products summed in
FP64, hidden and latent activations rounded to BF16 between the layers; the
GPU differs from it only by its FP32 accumulation order (and the rare BF16
rounding that order flips: one unit of the stored latent), so the bar is
tight (2e-3 of each row's largest value for the decoded rows, one BF16 unit
plus 1e-3 for the latents) and any error in the operand tiles, swizzle,
descriptors or epilogue indexing fails it.  (2) The FP64 oracle: the BF16 error is reported and held
to a loose bar (5e-2), as the precision reading allows.
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


def bf16_of_f32(a):
    """float32 -> nearest BF16 (ties to even), returned as float64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_of_f64(a):
    """float64 -> nearest BF16 (ties to even) in one rounding, as float64."""
    b = np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)
    sign = b & np.uint64(1 << 63)
    m = b & np.uint64(0x7FFFFFFFFFFFFFFF)
    m = m + np.uint64((1 << 44) - 1) + ((m >> np.uint64(45)) & np.uint64(1))
    m = m & ~np.uint64((1 << 45) - 1)
    return (m | sign).view(np.float64)


def act_np(act, v):
    return np.maximum(v, 0.0) if act == 1 else v


def emulate(p, x, act, tied):
    """The BF16 kernels' arithmetic in numpy (see the module docstring)."""
    f32 = np.float32
    W1, b1, W2, b2 = p["W1"], p["b1"], p["W2"], p["b2"]
    W3 = W2.T if tied else p["W3"]
    W4 = W1.T if tied else p["W4"]
    mu, sig = f32(p["mu"]), f32(p["sigma"])
    W1f = f32(W1) / sig[:, None]                      # [P][H], FP32 like the weight folding
    b1f = f32(f32(p["b1"]) - (W1f.astype(np.float64) * mu[:, None]).sum(axis=0))
    s = x.max(axis=1)
    rs = np.where(s > 0, f32(1.0 / s), f32(0.0)).astype(np.float64)
    acc = bf16_of_f64(x) @ bf16_of_f32(W1f)
    h = bf16_of_f32(f32(act_np(act, f32(acc * rs[:, None] + b1f))))
    z = bf16_of_f32(f32(h @ bf16_of_f32(f32(W2)) + f32(b2)))
    h3 = bf16_of_f32(f32(act_np(act, f32(z @ bf16_of_f32(f32(W3)) + f32(p["b3"])))))
    W4f = f32(sig[None, :] * f32(W4))                 # [H][P]
    b4f = f32(sig * f32(p["b4"]) + mu)
    xh = f32(s)[:, None].astype(np.float64) * f32(h3 @ bf16_of_f32(W4f) + b4f)
    return z, xh, s


def rand_params(P, H, L, tied, seed):
    d = synth.ae_init(P, H, L, seed, tied=tied)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3", "b4"):
        d[k] = rng.normal(0, 0.1, size=d[k].shape)
    d["mu"] = rng.uniform(0, 0.3, size=P)
    d["sigma"] = rng.uniform(0.5, 1.5, size=P)
    return d


@pytest.mark.parametrize("H,L,tied,act,sizes", [
    (256, 32, True, 0, [300]),
    (128, 16, False, 1, [5, 0, 130, 257]),
    (512, 32, True, 0, [129]),
])
def test_bf16_encode_decode(aq, H, L, tied, act, sizes):
    P = 1521
    G = len(sizes)
    m = aq.Model(P, H, L, tied=tied, act=act, dtype=aq.DTYPE_BF16, n_groups=G)
    prms = []
    for g in range(G):
        d = rand_params(P, H, L, tied, 70 + g)
        m.set_group(g, d)
        prms.append(d)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = synth.histograms(int(off[-1]), synth.config_seed(1) + H)
    goff = dev(off) if G > 1 else None
    z, s = aq.ae_encode(m, dev(x), group_offsets=goff)
    assert z.dtype == torch.bfloat16
    xh = aq.ae_decode(m, z, s, group_offsets=goff)
    torch.cuda.synchronize()
    z = z.float().cpu().numpy().astype(np.float64)
    s, xh = s.cpu().numpy(), xh.cpu().numpy()[:, :P].astype(np.float64)
    assert np.array_equal(s, x.max(axis=1))
    worst = {"latent": 0.0, "xhat": 0.0}
    for g in range(G):
        r = slice(off[g], off[g + 1])
        if sizes[g] == 0:
            continue
        ze, xe, _ = emulate(prms[g], x[r], act, tied)
        zsc = np.abs(ze).max(axis=1, keepdims=True) + 1e-30
        xsc = np.abs(xe).max(axis=1, keepdims=True) + 1e-30
        # the latent is stored in BF16: a different FP32 summation order may
        # flip its rounding by one unit (at most 2^-7 of the value)
        assert np.all(np.abs(z[r] - ze) <= 2.0 ** -7 * np.abs(ze) + 1e-3 * zsc)
        # the decoder reads the GPU's latents: compare against the emulation
        # of the decoder on those
        _, xe2, _ = emulate_decoder(prms[g], z[r], s[r], act, tied)
        assert np.all(np.abs(xh[r] - xe2) <= 2e-3 * xsc)
        zo, xo, so = oracle.ae_forward(oracle.AE(act=act, **prms[g]), x[r])
        worst["latent"] = max(worst["latent"], float((np.abs(z[r] - zo) / (np.abs(zo).max(
            axis=1, keepdims=True) + 1e-30)).max()))
        worst["xhat"] = max(worst["xhat"], float((np.abs(xh[r] - xo) / so[:, None]).max()))
    print("BF16 vs FP64 oracle, worst relative error:", worst)
    assert worst["latent"] < 5e-2 and worst["xhat"] < 5e-2


def emulate_decoder(p, z, s, act, tied):
    f32 = np.float32
    W1, W2 = p["W1"], p["W2"]
    W3 = W2.T if tied else p["W3"]
    W4 = W1.T if tied else p["W4"]
    mu, sig = f32(p["mu"]), f32(p["sigma"])
    h3 = bf16_of_f32(f32(act_np(act, f32(z @ bf16_of_f32(f32(W3)) + f32(p["b3"])))))
    W4f = f32(sig[None, :] * f32(W4))
    b4f = f32(sig * f32(p["b4"]) + mu)
    xh = f32(s)[:, None].astype(np.float64) * f32(h3 @ bf16_of_f32(W4f) + b4f)
    return z, xh, s


def test_bf16_shapes_outside_the_tensor_core_path_are_refused(aq):
    with pytest.raises(RuntimeError, match="BF16 models need"):
        aq.Model(1521, 96, 32, dtype=aq.DTYPE_BF16)


@pytest.mark.parametrize("H,L,tied,sizes", [
    (512, 32, True, [152 * 128 * 3 + 77]),          # three or four tiles per CTA
    (256, 32, True, [9000, 0, 31000, 1, 18000]),    # tiles of several groups per CTA
])
def test_bf16_persistent_tiles(aq, H, L, tied, sizes):
    """The persistent encoder and decoder (one CTA per SM walking the tiles):
    batches of several tiles per CTA, ungrouped and grouped, against the
    BF16 emulation on sampled rows of every group (first, last and evenly
    spaced rows, so every CTA's later tiles are among them)."""
    P = 1521
    G = len(sizes)
    m = aq.Model(P, H, L, tied=tied, act=0, dtype=aq.DTYPE_BF16, n_groups=G)
    prms = []
    for g in range(G):
        d = rand_params(P, H, L, tied, 90 + g)
        m.set_group(g, d)
        prms.append(d)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    xd = synth.histograms_torch(n, synth.config_seed(2) + H, DEV)
    goff = dev(off) if G > 1 else None
    z, s = aq.ae_encode(m, xd, group_offsets=goff)
    xh = aq.ae_decode(m, z, s, group_offsets=goff)
    torch.cuda.synchronize()
    for g in range(G):
        if sizes[g] == 0:
            continue
        rows = np.unique(np.concatenate([np.linspace(off[g], off[g + 1] - 1, 97),
                                         [off[g], off[g + 1] - 1]]).astype(np.int64))
        idx = torch.as_tensor(rows, device=DEV)
        x = xd[idx].cpu().numpy()
        zg = z[idx].float().cpu().numpy().astype(np.float64)
        sg = s[idx].cpu().numpy()
        xg = xh[idx].cpu().numpy()[:, :P].astype(np.float64)
        assert np.array_equal(sg, x.max(axis=1))
        ze, _, _ = emulate(prms[g], x, 0, tied)
        zsc = np.abs(ze).max(axis=1, keepdims=True) + 1e-30
        assert np.all(np.abs(zg - ze) <= 2.0 ** -7 * np.abs(ze) + 1e-3 * zsc), g
        _, xe, _ = emulate_decoder(prms[g], zg, sg, 0, tied)
        xsc = np.abs(xe).max(axis=1, keepdims=True) + 1e-30
        assert np.all(np.abs(xg - xe) <= 2e-3 * xsc), g


def test_bf16_input_rounding_is_nearest_even(aq):
    """The encoder's FP64 -> BF16 rounding of its input, seen through an
    identity first layer and a second layer that selects 16 of its 64 hidden
    units: with max(x) = 1 in every row (so 1/s = 1), latent l of row r is
    exactly BF16(x[r, 4 l]).  The inputs hold BF16 ties, values one FP64 unit
    either side of a tie, ties broken only by bits of the low 32-bit word,
    zeros, negative and tiny (but float-normal) values, and random doubles."""
    P = H = 64
    L = 16
    sel = np.arange(L) * 4
    W2 = np.zeros((H, L))
    W2[sel, np.arange(L)] = 1.0
    p = dict(W1=np.eye(P), b1=np.zeros(H), W2=W2, b2=np.zeros(L), W3=np.zeros((L, H)),
             b3=np.zeros(H), W4=np.zeros((H, P)), b4=np.zeros(P), mu=np.zeros(P),
             sigma=np.ones(P))
    m = aq.Model(P, H, L, tied=False, dtype=aq.DTYPE_BF16)
    m.set_group(0, p)
    rng = np.random.default_rng(11)
    n = 4096
    x = rng.uniform(0.0, 1.0, size=(n, P))
    # BF16 values b in [2^-40, 1) and their half-unit ties
    e = rng.integers(-40, 0, size=(n, L)).astype(np.float64)
    b = np.ldexp(1.0 + rng.integers(0, 128, size=(n, L)) / 128.0, e.astype(int) - 1)
    half = np.ldexp(1.0, e.astype(int) - 9)  # half a BF16 unit at b's binade
    kind = rng.integers(0, 8, size=(n, L))
    v = x[:, sel].copy()
    v[kind == 0] = (b + half)[kind == 0]                                  # tie
    v[kind == 1] = np.nextafter(b + half, np.inf)[kind == 1]              # just above
    v[kind == 2] = np.nextafter(b + half, 0.0)[kind == 2]                 # just below
    v[kind == 3] = (b + half * (1.0 + 2.0 ** -40))[kind == 3]             # low-word sticky bit
    v[kind == 4] = 0.0
    v[kind == 5] = -x[:, sel][kind == 5]
    v[kind == 6] = np.ldexp(0.5 + 0.5 * x[:, sel], -100)[kind == 6]       # tiny, float-normal
    x[:, sel] = v
    x[:, P - 1] = 1.0
    z, s = aq.ae_encode(m, dev(x))
    torch.cuda.synchronize()
    assert np.all(s.cpu().numpy() == 1.0)
    got = z.float().cpu().numpy().astype(np.float64)
    want = bf16_of_f64(x[:, sel])
    bad = np.argwhere(got != want)
    assert bad.size == 0, (bad[:5], x[:, sel][tuple(bad[0])], got[tuple(bad[0])],
                           want[tuple(bad[0])])
    m.close()
