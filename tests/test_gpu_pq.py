"""Product quantisation of the latents on the GPU against the oracle
(Sec. III Stage 3, Sec. V-B).

* The start table (no iteration) equals the oracle's bit for bit.
* Given a table, the codes equal the oracle's nearest-centroid decisions bit
  for bit (both in float32, ties to the lowest index), and decoding equals the
  table lookup.
* After Lloyd iterations the tables agree within the fixed-point resolution
  of the sums plus one float32 rounding, per subdomain, with ragged and empty
  subdomains, non-finite latents and bfloat16 latents.
* The whole pipeline with PQ'd latents (encode, quantise the latents, decode
  from the table, quantise the residual, correct) keeps every point within
  the bound and the moments to 1e-10."""
import numpy as np
import pytest

from oracle import pq as opq
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


def latents(n, L, seed):
    rng = np.random.default_rng(seed)
    scale = np.exp(rng.uniform(-3, 3, L))
    z = rng.standard_normal((n, L)) * scale + rng.uniform(-2, 2, L) * scale
    # a few clumps so that K-means has structure
    z[: n // 4] = np.round(z[: n // 4] / scale * 2) * scale / 2
    return z.astype(np.float32)


def table_tol(z, c):
    # fixed-point resolution of the sums (2^-62 of max|z| times the row
    # count) plus one float32 rounding of each centroid
    amax = np.nanmax(np.abs(np.where(np.isfinite(z), z, 0)), axis=0)[:, None]
    return amax * 2.0 ** (-62 + np.ceil(np.log2(max(len(z), 2)))) * 4 + np.spacing(np.abs(c))


@pytest.mark.parametrize("k", [16, 64, 256])
def test_start_table_and_codes_bit_exact(aq, k):
    n, L = 5000, 32
    z = latents(n, L, 1)
    zd = torch.as_tensor(z, device=DEV)
    t0 = aq.pq_train(zd, k=k, iters=0)
    np.testing.assert_array_equal(t0.cpu().numpy()[0], opq.init_centroids(z, k))
    ref = opq.train(z, k, 3)
    tab = torch.as_tensor(ref[None], device=DEV)
    zq = torch.empty_like(zd)
    codes, _ = aq.pq_encode(zd, tab, zq=zq)
    torch.cuda.synchronize()
    oc = opq.assign(z, ref)
    np.testing.assert_array_equal(codes.cpu().numpy(), oc)
    np.testing.assert_array_equal(zq.cpu().numpy(), opq.decode(oc, ref))
    dec = aq.pq_decode(codes, tab, torch.float32)
    np.testing.assert_array_equal(dec.cpu().numpy(), opq.decode(oc, ref))


@pytest.mark.parametrize("iters", [1, 10])
def test_lloyd_tables_match_oracle(aq, iters):
    n, L, k = 20000, 16, 16
    z = latents(n, L, 2)
    t = aq.pq_train(torch.as_tensor(z, device=DEV), k=k, iters=iters).cpu().numpy()[0]
    ref = opq.train(z, k, iters)
    if iters == 1:  # same start, same decisions: only the mean's rounding differs
        assert np.all(np.abs(t - ref) <= table_tol(z, ref))
    else:  # later decisions may flip at exact midpoints; the quantiser is as good
        codes = opq.assign(z, t)
        jg = opq.objective(z, codes, t)
        jo = opq.objective(z, opq.assign(z, ref), ref)
        assert abs(jg - jo) <= 1e-6 * jo
        assert np.mean(np.abs(t - ref) <= table_tol(z, ref)) > 0.99


def test_groups_ragged_empty_nonfinite_and_bf16(aq):
    L, k = 8, 16
    sizes = [3000, 0, 17, 1200]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    z = latents(int(off[-1]), L, 3)
    z[5, 2] = np.nan
    z[3010, 0] = np.inf
    zb = torch.as_tensor(z, device=DEV).to(torch.bfloat16)
    zf = zb.float().cpu().numpy()  # the values the GPU sees
    goff = torch.as_tensor(off, device=DEV)
    G = len(sizes)
    t = aq.pq_train(zb, k=k, iters=1, group_offsets=goff, G=G).cpu().numpy()
    ref = opq.train_grouped(zf, off, k, 1)
    for g in range(G):
        zg = zf[off[g]:off[g + 1]]
        if len(zg) == 0:
            np.testing.assert_array_equal(t[g], 0.0)
            continue
        assert np.all(np.abs(t[g] - ref[g]) <= table_tol(zg, ref[g])), g
    tab = torch.as_tensor(ref, device=DEV)
    zq = torch.empty_like(zb)
    codes, _ = aq.pq_encode(zb, tab, group_offsets=goff, zq=zq)
    torch.cuda.synchronize()
    for g in range(G):
        zg = zf[off[g]:off[g + 1]]
        oc = opq.assign(zg, ref[g])
        np.testing.assert_array_equal(codes.cpu().numpy()[off[g]:off[g + 1]], oc)
        want = torch.as_tensor(opq.decode(oc, ref[g])).to(torch.bfloat16).float().numpy()
        np.testing.assert_array_equal(zq.float().cpu().numpy()[off[g]:off[g + 1]], want)
    assert codes[5, 2].item() == 0 and codes[3010, 0].item() == 0


def test_argument_checks(aq):
    z = torch.zeros((10, 4), device=DEV)
    for bad in (dict(k=1), dict(k=257), dict(iters=-1)):
        with pytest.raises(aq.AeqcError):
            aq.pq_train(z, **{**dict(k=16, iters=1), **bad})
    with pytest.raises(aq.AeqcError):
        aq.pq_train(z, k=16, iters=1, G=2)  # G > 1 without offsets


def test_pipeline_with_pq_latents_keeps_the_bounds(aq):
    P, H, L, n, tau = 1521, 128, 16, 4000, 1e-4
    x = torch.as_tensor(synth.histograms(n, synth.config_seed(1) + 5), device=DEV)
    m = aq.Model(P, H, L, dtype=aq.DTYPE_BF16)
    m.set_group(0, synth.ae_init(P, H, L, 21))
    m.fit_normalizer(0, x[:512])
    ws = None
    for t in range(60):
        ws = m.train_step(x[(t * 64) % 3900:(t * 64) % 3900 + 64], lr=2e-3, ws=ws)
    z, s = aq.ae_encode(m, x)
    tab = aq.pq_train(z, k=16, iters=10)
    codes, _ = aq.pq_encode(z, tab, zq=z)  # z now holds the decoded latents
    xhat = aq.ae_decode(m, z, s)
    grid = aq.Grid(*synth.grid_arrays())
    p = aq.params_default(tau=tau, kernel=aq.KERNEL_FAST)
    out = aq.quantize_correct(grid, x, xhat, p, want_f=True, outlier_capacity=64 * P)
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()
    ok = (st & aq.ST_VERBATIM) == 0
    assert ok.mean() > 0.99
    f, xx = out.f.cpu().numpy()[ok], x.cpu().numpy()[ok]
    e = tau * xx.max(axis=1, keepdims=True)
    assert np.all(np.abs(f - xx) <= e)
    vpar, vperp, vol = synth.grid_arrays()
    V, W = np.meshgrid(vpar, vperp)
    phi = np.stack([np.ones(P), V.ravel(), W.ravel() ** 2, V.ravel() ** 2])
    qf, qx = f @ phi.T * vol, xx @ phi.T * vol
    sk = np.abs(xx) @ np.abs(phi).T * vol
    assert np.max(np.abs(qf - qx) / sk) <= 1e-10
