"""Incremental training across time steps (Sec. IV-B, Paradigm 3): the model
of the previous step, trained a few more steps on drifted data, fits that
data better than a fresh model with the same budget, and a checkpoint of it
resumes training exactly."""
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


def train(m, x, steps, B=64):
    ws = None
    for t in range(steps):
        i0 = (t * B) % (x.shape[0] - B)
        ws = m.train_step(x[i0:i0 + B], lr=1e-3, ws=ws)


def test_incremental_beats_fresh_on_drifted_step(aq):
    P, H, L, n = 1521, 64, 16, 4096
    x0 = torch.as_tensor(synth.histograms(n, 77, step=0), device=DEV)
    x1 = torch.as_tensor(synth.histograms(n, 77, step=1), device=DEV)
    m = aq.Model(P, H, L)
    m.set_group(0, synth.ae_init(P, H, L, 1))
    m.fit_normalizer(0, x0[:1024])
    train(m, x0, 400)
    train(m, x1, 40)
    f = aq.Model(P, H, L)
    f.set_group(0, synth.ae_init(P, H, L, 2))
    f.fit_normalizer(0, x1[:1024])
    train(f, x1, 40)
    # reconstruction error in data space (the two models normalise differently)
    ev = x1[-512:]

    def err(model):
        z, s = aq.ae_encode(model, ev)
        xh = aq.ae_decode(model, z, s)[:, :P].double()
        return ((xh - ev).norm() / ev.norm()).item()

    assert err(m) < 0.5 * err(f)
    # resume from a checkpoint: the next steps agree bit for bit
    c = aq.Model.load(m.save())
    train(m, x1, 5)
    train(c, x1, 5)
    assert m.save() == c.save()
