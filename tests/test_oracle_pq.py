"""Pins of the product-quantisation oracle (Sec. III Stage 3, Sec. V-B) against
facts of K-means that do not come from the oracle itself."""
import numpy as np
import pytest

from oracle import pq


def test_separated_clusters_give_their_means():
    # k groups far apart, membership known by construction
    rng = np.random.default_rng(1)
    k, per = 4, 500
    centers = np.array([-150.0, -50.0, 50.0, 150.0])
    cols = []
    truth = np.zeros((2, k))
    for d in range(2):
        vals, labels = [], []
        for j in range(k):
            v = (centers[j] * (d + 1) + rng.uniform(-1, 1, per)).astype(np.float32)
            vals.append(v)
            truth[d, j] = np.float32(np.sum(v.astype(np.float64)) / per)
        cols.append(np.concatenate(vals))
    z = np.stack(cols, axis=1)
    perm = rng.permutation(z.shape[0])
    z = z[perm]
    c = pq.train(z, k, 3)
    np.testing.assert_array_equal(c, truth.astype(np.float32))


def test_k_equally_spaced_values_are_reproduced_exactly():
    for k in (2, 4, 16):
        z = np.tile(np.arange(k, dtype=np.float32)[:, None], (7, 3))
        c = pq.train(z, k, 1)
        codes = pq.assign(z, c)
        np.testing.assert_array_equal(pq.decode(codes, c), z)
        assert pq.objective(z, codes, c) == 0.0


def test_assignment_is_the_nearest_centroid_brute_force():
    rng = np.random.default_rng(2)
    # values and centroids on dyadic grids: float32 distances are exact
    z = (rng.integers(-400, 400, size=(300, 3)) / 8.0).astype(np.float32)
    c = (np.sort(rng.integers(-64, 64, size=(3, 16)), axis=1) / 2.0).astype(np.float32)
    codes = pq.assign(z, c)
    for i in range(z.shape[0]):
        for d in range(3):
            dists = [abs(float(z[i, d]) - float(c[d, j])) for j in range(16)]
            best = min(dists)
            assert codes[i, d] == dists.index(best)  # lowest index on ties


def test_ties_go_to_the_lower_index():
    z = np.array([[1.0], [3.0]], dtype=np.float32)
    c = np.array([[0.0, 2.0, 4.0]], dtype=np.float32)
    np.testing.assert_array_equal(pq.assign(z, c)[:, 0], [0, 1])


def test_lloyd_objective_never_increases():
    rng = np.random.default_rng(3)
    z = rng.standard_normal((2000, 4)).astype(np.float32) * np.array([1, 5, 0.1, 30],
                                                                     dtype=np.float32)
    c = pq.init_centroids(z, 16)
    prev = pq.objective(z, pq.assign(z, c), c)
    for _ in range(8):
        c = pq.update(z, pq.assign(z, c), c)
        cur = pq.objective(z, pq.assign(z, c), c)
        assert cur <= prev * (1 + 1e-6)
        prev = cur


def test_empty_cluster_keeps_its_centroid_and_fixed_point():
    z = np.array([[0.0], [0.0], [10.0]], dtype=np.float32)
    c = np.array([[0.0, 10.0, 1000.0]], dtype=np.float32)
    c2 = pq.update(z, pq.assign(z, c), c)
    np.testing.assert_array_equal(c2, c)  # members at their centroids; 1000 is empty


def test_start_spans_the_column_range():
    z = np.array([[-2.0, 5.0], [6.0, 5.0]], dtype=np.float32)
    c = pq.init_centroids(z, 4)
    np.testing.assert_allclose(c[0], [-1.0, 1.0, 3.0, 5.0])
    np.testing.assert_array_equal(c[1], [5.0] * 4)  # constant column


@pytest.mark.parametrize("k", [16, 64])
def test_quantisation_error_shrinks_with_k(k):
    rng = np.random.default_rng(4)
    z = rng.standard_normal((3000, 2)).astype(np.float32)
    c = pq.train(z, k, 10)
    err = pq.objective(z, pq.assign(z, c), c) / z.size
    # uniform-quantiser scale: the mean squared error of k levels on N(0, 1)
    # is below the variance divided by ~k (loose bound, any sane K-means meets it)
    assert err < 4.0 / k
