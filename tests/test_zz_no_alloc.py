"""quantize_correct_noalloc (static device scratch, no workspace argument)
against quantize_correct (caller workspace) on the same inputs.

Both run the same kernels, so every output must agree exactly; the inputs
plant rows the fast kernel hands to the FP64 kernel (non-finite and negative
inputs, a zero image, non-finite decoded values), so the scratch list is
used.  Two calls in a row, the second smaller than the first, show that the
shared scratch carries nothing from one call into the next.
"""
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


def _batch(n, seed):
    x = synth.histograms(n, synth.config_seed(0) + seed)
    xh = synth.stand_in_xhat(x, seed)
    xh[0, 10] = np.nan
    xh[0, 11] = np.inf
    x[1, 5] = -1.0
    x[2, :] = 0.0
    x[3, 7] = np.nan
    return (torch.as_tensor(x, device=DEV), torch.as_tensor(np.ascontiguousarray(xh), device=DEV))


def _bits(t):
    """Bit patterns, so that NaNs stored verbatim compare equal."""
    return t.view(torch.int64) if t.dtype == torch.float64 else t


def _same(a, b):
    for name in ("codes", "scale", "lam", "iters", "status", "count", "f"):
        assert torch.equal(_bits(getattr(a, name)), _bits(getattr(b, name))), name
    # the outlier list is appended to atomically: compare it in index order
    k = int(a.count.item())
    ia, oa = torch.sort(a.index[:k])
    ib, ob = torch.sort(b.index[:k])
    assert torch.equal(ia, ib)
    assert torch.equal(_bits(a.value[:k][oa]), _bits(b.value[:k][ob]))


@pytest.mark.parametrize("kernel", ["fast", "fp64"])
def test_noalloc_matches_workspace_call_twice(aq, kernel):
    vpar, vperp, vol = synth.grid_arrays()
    grid = aq.Grid(vpar, vperp, vol)
    k = aq.KERNEL_FAST if kernel == "fast" else aq.KERNEL_FP64
    p = aq.params_default(tau=1e-4, kernel=k)
    for n, seed in ((1501, 31), (257, 32)):
        x, xh = _batch(n, seed)
        ref = aq.quantize_correct(grid, x, xh, p, outlier_capacity=1 << 16, want_f=True)
        got = aq.quantize_correct_noalloc(grid, x, xh, p, outlier_capacity=1 << 16, want_f=True)
        torch.cuda.synchronize()
        _same(ref, got)
        st = got.status.cpu().numpy()
        assert st[2] & aq.ST_ZERO_IMAGE and st[1] & aq.ST_NONFINITE_INPUT
