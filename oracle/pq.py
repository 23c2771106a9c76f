"""Product quantisation of the latent space, plain numpy (test infrastructure).

Only the test suite and ``bench.py``'s CPU baseline may import this module; it
shares no code with the CUDA library.

Sec. III (Stage 3) and Sec. V-B: the latent vectors of one processor's
histograms are quantised column by column: K-means with k clusters in each of
the L latent dimensions, each value replaced by the index of its cluster
(log2 k bits) and decoded as that cluster's centroid (a float32 PQ table of
k x L entries per processor).  The paper does not state the K-means start or
the number of iterations.  Readings:

* start: k centroids evenly spaced inside the column's range,
  c_j = lo + (j + 1/2) (hi - lo) / k in float64, rounded to float32;
* one Lloyd iteration = assign every value to its nearest centroid, then move
  each centroid to the mean of its members (float64 mean, rounded to float32);
  a centroid without members stays where it is;
* nearest = smallest |z - c_j| evaluated in float32 (the latents are float32
  or bfloat16), ties to the lowest index;
* each subdomain (group) has its own table;
* a non-finite latent value takes no part in training (range and means) and
  encodes as index 0 (no distance is smaller than a NaN's first one).

Pins (tests/test_oracle_pq.py): Lloyd's objective never increases; data drawn
from k separated clusters gives the clusters' means exactly; k at least the
number of distinct values gives zero error; assignments equal a brute-force
nearest search; a single value per cluster is a fixed point.
"""
from __future__ import annotations

import numpy as np


def init_centroids(z: np.ndarray, k: int) -> np.ndarray:
    """[L][k] float32 start: k points evenly spaced in each column's range."""
    z = np.asarray(z, dtype=np.float32)
    L = z.shape[1]
    c = np.zeros((L, k), dtype=np.float32)
    if z.shape[0] == 0:
        return c
    for d in range(L):
        col = z[:, d][np.isfinite(z[:, d])]
        if col.size == 0:
            continue
        lo = float(np.min(col))
        hi = float(np.max(col))
        for j in range(k):
            c[d, j] = np.float32(lo + (j + 0.5) * (hi - lo) / k)
    return c


def assign(z: np.ndarray, c: np.ndarray) -> np.ndarray:
    """codes [n][L] uint8: index of the nearest centroid per value (float32
    distances, lowest index on ties)."""
    z = np.asarray(z, dtype=np.float32)
    n, L = z.shape
    k = c.shape[1]
    codes = np.zeros((n, L), dtype=np.uint8)
    for d in range(L):
        best = np.full(n, np.inf, dtype=np.float32)
        arg = np.zeros(n, dtype=np.int64)
        for j in range(k):
            dist = np.abs(z[:, d] - np.float32(c[d, j]))  # float32 arithmetic
            better = dist < best
            best = np.where(better, dist, best)
            arg = np.where(better, j, arg)
        codes[:, d] = arg
    return codes


def update(z: np.ndarray, codes: np.ndarray, c: np.ndarray) -> np.ndarray:
    """New centroids: the float64 mean of each cluster's members, rounded to
    float32; empty clusters keep their centroid."""
    z = np.asarray(z, dtype=np.float32)
    L, k = c.shape
    out = c.copy()
    for d in range(L):
        fin = np.isfinite(z[:, d])
        for j in range(k):
            m = (codes[:, d] == j) & fin
            cnt = int(np.count_nonzero(m))
            if cnt:
                out[d, j] = np.float32(np.sum(z[m, d].astype(np.float64)) / cnt)
    return out


def train(z: np.ndarray, k: int, iters: int) -> np.ndarray:
    """[L][k] PQ table after `iters` Lloyd iterations from init_centroids."""
    c = init_centroids(z, k)
    for _ in range(iters):
        c = update(z, assign(z, c), c)
    return c


def decode(codes: np.ndarray, c: np.ndarray) -> np.ndarray:
    """[n][L] float32 latents from codes and the table."""
    n, L = codes.shape
    out = np.zeros((n, L), dtype=np.float32)
    for d in range(L):
        out[:, d] = c[d, codes[:, d].astype(np.int64)]
    return out


def objective(z: np.ndarray, codes: np.ndarray, c: np.ndarray) -> float:
    """Sum of squared quantisation errors (float64)."""
    zq = decode(codes, c).astype(np.float64)
    return float(np.sum((np.asarray(z, dtype=np.float64) - zq) ** 2))


def train_grouped(z: np.ndarray, offsets, k: int, iters: int) -> np.ndarray:
    """[G][L][k]: one table per group of rows [offsets[g], offsets[g+1])."""
    G = len(offsets) - 1
    L = z.shape[1]
    out = np.zeros((G, L, k), dtype=np.float32)
    for g in range(G):
        out[g] = train(z[offsets[g]:offsets[g + 1]], k, iters)
    return out
