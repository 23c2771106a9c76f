"""compress_batch_host (host memory in and out, chunked, copies overlapped
with compute) gives the same results as compress_batch on the whole batch in
device memory: latents, scales, codes, multipliers, iterations and statuses
bit for bit, the outlier lists equal as sets of (global index, value)."""
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


@pytest.mark.parametrize("dtype,H,L,kernel,chunk", [
    ("f32", 64, 16, "fast", 2048),
    ("bf16", 128, 16, "fast", 1536),
    ("f32", 64, 16, "fp64", 4096),
])
def test_host_stream_matches_device_batch(aq, dtype, H, L, kernel, chunk):
    P, n = 1521, 5000
    x = synth.histograms(n, synth.config_seed(1) + 55)
    # two histograms stored verbatim (every point an outlier), in different chunks
    x[7, 5] = np.nan
    x[4000, 9] = -1.0
    xd = torch.as_tensor(x, device=DEV)
    m = aq.Model(P, H, L, dtype=aq.DTYPE_BF16 if dtype == "bf16" else aq.DTYPE_F32)
    m.set_group(0, synth.ae_init(P, H, L, 9))   # untrained: large residuals
    m.fit_normalizer(0, xd[8:72])
    grid = aq.Grid(*synth.grid_arrays())
    p = aq.params_default(tau=1e-4, kernel=aq.KERNEL_FAST if kernel == "fast" else aq.KERNEL_FP64)
    cap = 4 * P
    ref = aq.compress_batch(m, grid, xd, p, outlier_capacity=cap)
    xh = torch.empty(x.shape, dtype=torch.float64, pin_memory=True)
    xh.copy_(torch.as_tensor(x))
    got = aq.compress_batch_host(m, grid, xh, p, chunk=chunk, outlier_capacity=cap)
    torch.cuda.synchronize()
    for k in ("latent", "scale", "codes", "lam", "iters", "status"):
        a, b = getattr(ref, k).cpu(), getattr(got, k)
        # bit patterns: the verbatim rows carry NaNs
        bits = {torch.float64: torch.int64, torch.float32: torch.int32,
                torch.bfloat16: torch.int16}
        if a.dtype in bits:
            a, b = a.view(bits[a.dtype]), b.view(bits[a.dtype])
        assert torch.equal(a, b), k
    cnt = int(ref.count.item())
    assert cnt == int(got.count.item()) and cnt >= 2 * P
    ia, oa = torch.sort(ref.index[:cnt].cpu())
    ib, ob = torch.sort(got.index[:cnt])
    assert torch.equal(ia, ib)
    assert torch.equal(ref.value[:cnt].cpu()[oa].view(torch.int64), got.value[:cnt][ob].view(torch.int64))
