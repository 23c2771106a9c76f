"""Launch tuning, the autotuner and CUDA-graph capture of compress_batch.

Launch choices change speed only: outputs must be bit-identical for every
tuning, for the autotuner's choice, and for a captured-and-replayed graph
of the same call (grouped batch with an empty group and ragged groups)."""
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


@pytest.fixture(scope="module")
def setup(aq):
    P, H, L = 1521, 128, 16
    sizes = [700, 0, 129, 1000]
    G = len(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = torch.as_tensor(synth.histograms(int(off[-1]), synth.config_seed(3) + 11), device=DEV)
    m = aq.Model(P, H, L, dtype=aq.DTYPE_BF16, n_groups=G)
    for g in range(G):
        m.set_group(g, synth.ae_init(P, H, L, 300 + g))
        if sizes[g]:
            m.fit_normalizer(g, x[off[g]:off[g + 1]])
    grid = aq.Grid(*synth.grid_arrays())
    p = aq.params_default(tau=1e-4, kernel=aq.KERNEL_FAST)
    return m, grid, p, x, torch.as_tensor(off, device=DEV)


def outputs(out):
    bits = {torch.float64: torch.int64, torch.float32: torch.int32, torch.bfloat16: torch.int16}
    res = {}
    for k in ("latent", "scale", "codes", "lam", "iters", "status", "count"):
        t = getattr(out, k).clone()
        res[k] = t.view(bits[t.dtype]) if t.dtype in bits else t
    return res


def same(a, b):
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_tuning_roundtrip_and_validation(aq, setup):
    m = setup[0]
    m.set_tuning(enc_stages=3, dec_stages=2, qc_warps_per_sm=8)
    assert m.get_tuning() == dict(enc_stages=3, dec_stages=2, qc_warps_per_sm=8)
    for bad in (dict(enc_stages=1), dict(enc_stages=7), dict(dec_stages=17),
                dict(qc_warps_per_sm=5), dict(qc_warps_per_sm=20)):
        with pytest.raises(RuntimeError):
            m.set_tuning(**bad)
    m.set_tuning()
    assert m.get_tuning() == dict(enc_stages=0, dec_stages=0, qc_warps_per_sm=0)


def test_results_do_not_depend_on_tuning(aq, setup):
    m, grid, p, x, goff = setup
    ref = None
    for t in (dict(), dict(enc_stages=2, dec_stages=2, qc_warps_per_sm=4),
              dict(enc_stages=5, dec_stages=3, qc_warps_per_sm=12),
              dict(enc_stages=4, dec_stages=16, qc_warps_per_sm=8)):
        m.set_tuning(**t)
        out = aq.compress_batch(m, grid, x, p, group_offsets=goff, outlier_capacity=1 << 16)
        torch.cuda.synchronize()
        o = outputs(out)
        if ref is None:
            ref = o
        else:
            same(ref, o)
    m.set_tuning()


def test_autotune_choice_is_valid_and_exact(aq, setup):
    m, grid, p, x, goff = setup
    m.set_tuning()
    ref = outputs(aq.compress_batch(m, grid, x, p, group_offsets=goff, outlier_capacity=1 << 16))
    out = aq.Compressed(x.shape[0], 1521, m.L, m.latent_dtype(), x.device, 1 << 16)
    best = aq.autotune(m, grid, x, p, group_offsets=goff, out=out)
    torch.cuda.synchronize()
    assert 2 <= best["enc_stages"] <= 6 and 2 <= best["dec_stages"] <= 16
    assert best["qc_warps_per_sm"] in (4, 8, 12, 16)
    assert m.get_tuning() == best
    same(ref, outputs(out))
    m.set_tuning()


def test_cuda_graph_replay_matches_direct_call(aq, setup):
    m, grid, p, x, goff = setup
    n = x.shape[0]
    ref = outputs(aq.compress_batch(m, grid, x, p, group_offsets=goff, outlier_capacity=1 << 16))
    out = aq.Compressed(n, 1521, m.L, m.latent_dtype(), x.device, 1 << 16)
    ws = aq.compress_batch_workspace(m, n, x.device)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside the capture (one-time host set-up)
        aq.compress_batch(m, grid, x, p, group_offsets=goff, out=out, ws=ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for t in (out.codes, out.lam, out.status):
        t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        aq.compress_batch(m, grid, x, p, group_offsets=goff, out=out, ws=ws,
                          stream=torch.cuda.current_stream())
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    same(ref, outputs(out))
