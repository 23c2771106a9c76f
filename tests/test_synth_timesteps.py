"""The time-step drift of the synthetic inputs (incremental training
workload): step 0 is the plain workload bit for bit; later steps move the
mixture centres and scale the amplitudes as stated."""
import numpy as np

from paper_2212_10733_gb300 import synth


def test_step_zero_is_the_plain_workload():
    np.testing.assert_array_equal(synth.histograms(20, 11, step=0), synth.histograms(20, 11))


def test_drift_moves_centres_and_amplitudes():
    prm = synth.gaussian_params(50, 3)
    d = synth.drift_params(prm, 2)
    np.testing.assert_allclose(d["c_par"], prm["c_par"] + 0.1)
    np.testing.assert_allclose(d["c_perp"], prm["c_perp"] + 0.06)
    np.testing.assert_allclose(d["amp"], prm["amp"] * 1.02 ** 2)
    np.testing.assert_array_equal(d["s_par"], prm["s_par"])
    x0, x1 = synth.histograms(50, 3), synth.histograms(50, 3, step=1)
    assert not np.array_equal(x0, x1)
    # a small step: the histograms stay close
    assert np.max(np.abs(x1 - x0)) < 0.2 * np.max(x0)


def test_paper_grid_shape():
    # 37 v_par x 33 v_perp cells: P = 1221, v_perp = 0 row exactly zero,
    # the same velocity ranges as the 39 x 39 grid
    x = synth.histograms(5, 2, grid=(37, 33))
    assert x.shape == (5, 1221)
    assert np.all(x.reshape(5, 33, 37)[:, 0, :] == 0.0) and np.all(x >= 0.0)
    vpar, vperp, vol = synth.grid_arrays(37, 33)
    assert vpar[0] == -4.0 and vpar[-1] == 4.0 and vperp[-1] == 4.0
    assert abs(vol - (8.0 / 36) * (4.0 / 32)) < 1e-15
