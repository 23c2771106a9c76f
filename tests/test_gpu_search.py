"""NRMSE (Eq. (7)) on the GPU against the oracle, and the error-bound search:
the returned bound, compressed and decompressed again through the public
calls, meets the NRMSE target (measured by the oracle's Eq. (7)), the
reported NRMSE is that value, and the search lands near the target."""
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


def test_nrmse_matches_oracle(aq):
    rng = np.random.default_rng(1)
    x = synth.histograms(300, synth.config_seed(1) + 3)
    f = x + rng.normal(0, 1e-4, x.shape) * x.max(axis=1, keepdims=True)
    b, ph = aq.nrmse_batch(torch.as_tensor(x, device=DEV), torch.as_tensor(f, device=DEV),
                           per_hist=True)
    ph = ph.cpu().numpy()
    for i in range(0, 300, 37):
        want = oracle.nrmse(x[i], f[i])
        assert abs(ph[i] - want) <= 1e-13 * want
    want = oracle.nrmse(x, f)
    assert abs(b - want) <= 1e-12 * want


@pytest.fixture(scope="module")
def small(aq):
    P, H, L, n = 1521, 64, 16, 1500
    x = torch.as_tensor(synth.histograms(n, synth.config_seed(1) + 8), device=DEV)
    m = aq.Model(P, H, L)
    m.set_group(0, synth.ae_init(P, H, L, 5))
    m.fit_normalizer(0, x[:512])
    ws = None
    for t in range(40):
        ws = m.train_step(x[(t * 32) % 1400:(t * 32) % 1400 + 32], lr=2e-3, ws=ws)
    return m, aq.Grid(*synth.grid_arrays()), x


def test_bound_search_meets_target(aq, small):
    m, grid, x = small
    p = aq.params_default(tau=1e-4, kernel=aq.KERNEL_FAST)
    target = 2e-5
    tau, e = aq.bound_search(m, grid, x, p, target, tau_lo=1e-6, tau_hi=1e-2, probes=14,
                             outlier_capacity=x.numel())
    assert 1e-6 <= tau <= 1e-2 and e <= target and e >= 0.5 * target
    p2 = aq.params_default(tau=tau, kernel=aq.KERNEL_FAST)
    out = aq.compress_batch(m, grid, x, p2, outlier_capacity=x.numel())
    f = aq.decompress_batch(m, grid, out, p2)
    torch.cuda.synchronize()
    ref = oracle.nrmse(x.cpu().numpy(), f.cpu().numpy())
    assert ref <= target
    assert abs(ref - e) <= 1e-12 * ref


def test_bound_search_unreachable_target(aq, small):
    m, grid, x = small
    p = aq.params_default(kernel=aq.KERNEL_FAST)
    with pytest.raises(aq.AeqcError) as err:
        aq.bound_search(m, grid, x, p, 1e-12, tau_lo=1e-3, tau_hi=1e-1, probes=3)
    assert err.value.code == aq.EUNSUPPORTED
