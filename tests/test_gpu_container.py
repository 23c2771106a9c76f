"""Checkpoints and the batch container on the GPU.

* A model saved after some training steps and loaded back gives bit-identical
  compressed outputs, and one more training step from the loaded copy (its
  Adam moments and step count restored) gives the same parameters as the
  same step on the original.
* An MLP saved and loaded predicts the same multipliers bit for bit.
* A compressed batch packed into a container blob and unpacked into fresh
  device buffers decompresses to the same histograms bit for bit, verbatim
  rows and the outlier list included."""
import numpy as np
import pytest

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


def bits(t):
    m = {torch.float64: torch.int64, torch.float32: torch.int32, torch.bfloat16: torch.int16}
    return t.view(m[t.dtype]) if t.dtype in m else t


def same_outputs(a, b):
    for k in ("latent", "scale", "codes", "lam", "iters", "status", "count"):
        assert torch.equal(bits(getattr(a, k)), bits(getattr(b, k))), k


@pytest.mark.parametrize("dtype,H,L,G", [("f32", 64, 16, 1), ("bf16", 128, 16, 2)])
def test_model_checkpoint_roundtrip(aq, dtype, H, L, G):
    P, n = 1521, 1200
    x = torch.as_tensor(synth.histograms(n, synth.config_seed(2) + 77), device=DEV)
    m = aq.Model(P, H, L, dtype=aq.DTYPE_BF16 if dtype == "bf16" else aq.DTYPE_F32, n_groups=G)
    for g in range(G):
        m.set_group(g, synth.ae_init(P, H, L, 40 + g))
        m.fit_normalizer(g, x[:256])
    ws = None
    for t in range(3):
        ws = m.train_step(x[t * 128:(t + 1) * 128], lr=1e-3, group=G - 1, ws=ws)
    torch.cuda.synchronize()
    blob = m.save()
    m2 = aq.Model.load(blob)
    assert (m2.P, m2.H, m2.L) == (P, H, L)
    assert m2.save() == blob
    goff = torch.as_tensor([0] + [n // G * (g + 1) for g in range(G - 1)] + [n], device=DEV)
    grid = aq.Grid(*synth.grid_arrays())
    p = aq.params_default(tau=1e-4, kernel=aq.KERNEL_FAST)
    a = aq.compress_batch(m, grid, x, p, group_offsets=goff, outlier_capacity=1 << 16)
    b = aq.compress_batch(m2, grid, x, p, group_offsets=goff, outlier_capacity=1 << 16)
    torch.cuda.synchronize()
    same_outputs(a, b)
    # Adam state: the next step agrees
    m.train_step(x[512:640], lr=1e-3, group=G - 1)
    m2.train_step(x[512:640], lr=1e-3, group=G - 1)
    torch.cuda.synchronize()
    assert m.save() == m2.save()


def test_mlp_checkpoint_roundtrip(aq):
    nin = 20
    mlp = aq.MLP(nin, 64)
    rng = np.random.default_rng(5)
    mlp.set({**synth.mlp_init(nin, 64, 4, 3),
             "in_mu": rng.normal(size=nin), "in_sd": rng.uniform(0.5, 2, nin),
             "out_mu": rng.normal(size=4), "out_sd": rng.uniform(0.5, 2, 4)})
    inp = torch.as_tensor(rng.normal(size=(4096, nin)).astype(np.float32), device=DEV)
    tgt = torch.as_tensor(rng.normal(size=(4096, 4)), device=DEV)
    ws = None
    for t in range(4):
        ws = mlp.train_step(inp[t * 512:(t + 1) * 512], tgt[t * 512:(t + 1) * 512], ws=ws)
    torch.cuda.synchronize()
    blob = mlp.save()
    m2 = aq.MLP.load(blob)
    assert m2.n_in == nin and m2.nh == 64
    assert torch.equal(bits(mlp.predict(inp)), bits(m2.predict(inp)))
    mlp.train_step(inp[:512], tgt[:512])
    m2.train_step(inp[:512], tgt[:512])
    torch.cuda.synchronize()
    assert mlp.save() == m2.save()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batch_container_roundtrip(aq, dtype):
    P, H, L, n = 1521, 128, 16, 3000
    x = synth.histograms(n, synth.config_seed(1) + 91)
    x[11, 3] = np.nan        # verbatim rows: every point in the outlier list
    x[2500, 40] = -2.0
    xd = torch.as_tensor(x, device=DEV)
    m = aq.Model(P, H, L, dtype=aq.DTYPE_BF16 if dtype == "bf16" else aq.DTYPE_F32)
    m.set_group(0, synth.ae_init(P, H, L, 12))
    m.fit_normalizer(0, xd[100:400])
    grid = aq.Grid(*synth.grid_arrays())
    p = aq.params_default(tau=1e-4, kernel=aq.KERNEL_FAST)
    comp = aq.compress_batch(m, grid, xd, p, outlier_capacity=8 * P)
    torch.cuda.synchronize()
    cnt = int(comp.count.item())
    assert cnt >= 2 * P
    blob = aq.batch_pack(comp)
    hdr = aq.batch_peek(blob)
    assert hdr == dict(n=n, P=P, L=L, latent_dtype=m.desc.dtype, outliers=cnt)
    back = aq.batch_unpack(blob, DEV)
    torch.cuda.synchronize()
    same_outputs(comp, back)
    assert torch.equal(comp.index[:cnt], back.index[:cnt])
    assert torch.equal(bits(comp.value[:cnt]), bits(back.value[:cnt]))
    fa = aq.decompress_batch(m, grid, comp, p)
    fb = aq.decompress_batch(m, grid, back, p)
    torch.cuda.synchronize()
    assert torch.equal(bits(fa), bits(fb))
    # a flipped byte in the header is caught; in the payload it is not the
    # container's business (no checksum), so only the header is tested
    bad = bytearray(blob)
    bad[16] ^= 1   # n
    with pytest.raises(aq.AeqcError) as e:
        aq.batch_unpack(bytes(bad), DEV)
    assert e.value.code == aq.ECORRUPT
