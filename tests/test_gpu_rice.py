"""Golomb-Rice coding of the residual codes on the GPU against the oracle:
parameters, lengths, offsets and stream words bit for bit; round trips on the
codes of a real compression; edge cases (no histogram, short rows, every
symbol escaped, every point at the zero level); damaged streams and offsets
decode without leaving their buffers (wrong codes, no stray access)."""
import numpy as np
import pytest

from oracle import rice as orice
from paper_2212_10733_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"
ZERO, ESC = orice.ZERO_CODE, orice.ESCAPE


@pytest.fixture(scope="module")
def aq():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2212_10733_gb300 import aeqc
    aeqc.load()
    return aeqc


def mixed_codes(n, P, seed):
    rng = np.random.default_rng(seed)
    scales = np.exp(rng.uniform(np.log(0.2), np.log(3e4), n))[:, None]
    q = np.clip(np.rint(rng.laplace(0, 1, (n, P)) * scales), -32766, 32766).astype(np.int16)
    z = rng.random((n, P)) < 0.05
    q[z] = ZERO
    q[rng.random((n, P)) < 0.002] = ESC
    q[0, :] = ZERO          # every point at the zero level
    q[1, :] = ESC           # every symbol escaped (capped prefix)
    q[2, :] = 32766
    q[3, :] = 0
    return q


def check_against_oracle(aq, q):
    rs = aq.rice_encode(torch.as_tensor(q, device=DEV))
    torch.cuda.synchronize()
    ks, nb, off, words = orice.encode(q)
    np.testing.assert_array_equal(rs.kparam.cpu().numpy(), ks)
    np.testing.assert_array_equal(rs.nbits.cpu().numpy().astype(np.uint32), nb)
    np.testing.assert_array_equal(rs.offsets.cpu().numpy(), off)
    np.testing.assert_array_equal(rs.words.cpu().numpy().view(np.uint32), words)
    dec = aq.rice_decode(rs, q.shape[1])
    np.testing.assert_array_equal(dec.cpu().numpy(), q)


@pytest.mark.parametrize("P", [1521, 7, 1536])
def test_streams_bit_exact(aq, P):
    check_against_oracle(aq, mixed_codes(24, P, P))


def test_round_trip_real_codes(aq):
    P, H, L, n = 1521, 64, 16, 6000
    x = torch.as_tensor(synth.histograms(n, synth.config_seed(1) + 17), device=DEV)
    m = aq.Model(P, H, L)
    m.set_group(0, synth.ae_init(P, H, L, 3))
    m.fit_normalizer(0, x[:512])
    grid = aq.Grid(*synth.grid_arrays())
    out = aq.compress_batch(m, grid, x, aq.params_default(tau=1e-4, kernel=aq.KERNEL_FAST),
                            outlier_capacity=1 << 16)
    codes = out.codes
    rs = aq.rice_encode(codes)
    dec = aq.rice_decode(rs, P)
    torch.cuda.synchronize()
    assert torch.equal(dec, codes)
    # a sample against the oracle, bit for bit
    sample = codes[::1000].cpu().numpy()
    ks, nb, off, words = orice.encode(sample)
    np.testing.assert_array_equal(rs.kparam[::1000].cpu().numpy(), ks)
    np.testing.assert_array_equal(rs.nbits[::1000].cpu().numpy().astype(np.uint32), nb)
    o = rs.offsets.cpu().numpy()
    w = rs.words.cpu().numpy().view(np.uint32)
    for i, b in enumerate(range(0, n, 1000)):
        np.testing.assert_array_equal(w[o[b]:o[b + 1]], words[off[i]:off[i + 1]])


def test_empty_batch(aq):
    rs = aq.rice_encode(torch.empty((0, 1521), dtype=torch.int16, device=DEV))
    assert rs.offsets.cpu().tolist() == [0] and rs.words.numel() == 0
    assert aq.rice_decode(rs, 1521).shape == (0, 1521)


def test_damaged_streams_stay_in_bounds(aq):
    q = mixed_codes(64, 1521, 5)
    rs = aq.rice_encode(torch.as_tensor(q, device=DEV))
    g = torch.Generator(device="cpu").manual_seed(9)
    flips = torch.randint(0, 32, (rs.words.numel(),), generator=g).to(DEV)
    words = rs.words ^ (1 << flips).to(torch.int32)
    bad = aq.RiceStreams(rs.kparam, rs.nbits, rs.offsets, words)
    d1 = aq.rice_decode(bad, 1521)
    off = rs.offsets.clone()
    off[5] = 1 << 40          # beyond the words
    off[9] = -7               # before the words
    off[20] = off[30]         # overlapping
    d2 = aq.rice_decode(aq.RiceStreams(rs.kparam, rs.nbits, off, rs.words), 1521)
    torch.cuda.synchronize()
    assert d1.shape == d2.shape == (64, 1521)
    # histograms whose stream and offsets are intact still decode exactly
    ok = [b for b in range(64) if b not in (4, 5, 8, 9, 19, 20)]
    np.testing.assert_array_equal(d2.cpu().numpy()[ok], q[ok])
