"""Seeded synthetic inputs shaped like the paper's XGC velocity-space data.

This module holds none of the compression method's arithmetic: it only makes
inputs (the velocity grid, histograms, stand-in decoded histograms, subdomain
sizes, initial network weights) that both the CUDA path and the oracle
consume byte for byte.

The XGC ITER F-data the paper compresses (Sec. IV-A: 8 planes x 1.1e6 mesh
nodes x 33 x 37 velocity cells, values from 2.2e3 to 6.6e17) is not
available, so seeded stand-ins keep its structure: many small, positive 2D
histograms on a (v_perp, v_par) grid carrying the v_perp Jacobian factor,
grouped into subdomains of uneven size (Sec. III Stage 1).

Recipe (one numpy Philox stream per seed, draws in a fixed order):
  * grid: v_par_i = -4 + 8 i / 38, v_perp_j = 4 j / 38 (39 x 39), uniform cell
    volume (8/38)(4/38);
  * each histogram: K ~ U{1..k_max} Gaussians with amplitude ~ LogUniform[0.5, 2],
    centre v_par ~ U[-2, 2], v_perp ~ U[0.5, 2.5], widths ~ U[0.5, 1.5] each;
    x_ji = v_perp_j * sum_k amp_k exp(-(v_par_i - c_par)^2 / 2 s_par^2
                                      -(v_perp_j - c_perp)^2 / 2 s_perp^2);
  * heavy tail (optional): a fraction of histograms gets floor noise
    1e-6 * max(x) * |t_2| (Student t, 2 degrees of freedom, clipped at 1e3);
  * subdomain sizes: lognormal, median 8192, sigma_ln 0.85, clipped to
    [1024, 65536];
  * time steps (incremental training, Sec. IV-B): step t moves every centre
    by t * (drift_par, drift_perp) and scales every amplitude by
    (1 + drift_amp)^t, so consecutive steps are close but not equal.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2212_10733
N_PAR = 39
N_PERP = 39
P = N_PAR * N_PERP


def config_seed(config_index: int) -> int:
    return BASE_SEED + int(config_index)


def grid_arrays(n_par: int = N_PAR, n_perp: int = N_PERP, vpar_max: float = 4.0,
                vperp_max: float = 4.0):
    """v_par [n_par], v_perp [n_perp], uniform cell volume."""
    vpar = -vpar_max + 2.0 * vpar_max * np.arange(n_par, dtype=np.float64) / (n_par - 1)
    vperp = vperp_max * np.arange(n_perp, dtype=np.float64) / (n_perp - 1)
    vol = (2.0 * vpar_max / (n_par - 1)) * (vperp_max / (n_perp - 1))
    return vpar, vperp, float(vol)


def gaussian_params(n: int, seed: int, k_max: int = 3):
    """Per-histogram mixture parameters, each [n][k_max]; inactive terms have amp 0."""
    rng = np.random.Generator(np.random.Philox(seed))
    k = rng.integers(1, k_max + 1, size=n)
    amp = np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=(n, k_max)))
    c_par = rng.uniform(-2.0, 2.0, size=(n, k_max))
    c_perp = rng.uniform(0.5, 2.5, size=(n, k_max))
    s_par = rng.uniform(0.5, 1.5, size=(n, k_max))
    s_perp = rng.uniform(0.5, 1.5, size=(n, k_max))
    amp = np.where(np.arange(k_max)[None, :] < k[:, None], amp, 0.0)
    return dict(amp=amp, c_par=c_par, c_perp=c_perp, s_par=s_par, s_perp=s_perp)


def drift_params(prm: dict, t: int, drift_par: float = 0.05, drift_perp: float = 0.03,
                 drift_amp: float = 0.02) -> dict:
    """Mixture parameters of time step t (t = 0: unchanged)."""
    out = dict(prm)
    out["c_par"] = prm["c_par"] + t * drift_par
    out["c_perp"] = prm["c_perp"] + t * drift_perp
    out["amp"] = prm["amp"] * (1.0 + drift_amp) ** t
    return out


def _eval_numpy(prm, idx, vpar, vperp):
    a = {k: v[idx] for k, v in prm.items()}
    ea = np.exp(-(vpar[None, None, :] - a["c_par"][:, :, None]) ** 2
                / (2.0 * a["s_par"][:, :, None] ** 2))
    eb = np.exp(-(vperp[None, None, :] - a["c_perp"][:, :, None]) ** 2
                / (2.0 * a["s_perp"][:, :, None] ** 2))
    x = np.einsum("nk,nki,nkj->nji", a["amp"], ea, eb)
    return x * vperp[None, :, None]


def histograms(n: int, seed: int, k_max: int = 3, heavy_frac: float = 0.0,
               idx=None, step: int = 0, grid=(N_PAR, N_PERP)) -> np.ndarray:
    """Histograms [len(idx) or n][n_perp * n_par] float64 (i fastest).

    ``idx`` selects a subset of the n-histogram workload (same values as the
    full set at those indices); ``step`` is the time step (drift_params);
    ``grid`` = (n_par, n_perp) (the paper's XGC mesh nodes are 37 x 33)."""
    vpar, vperp, _ = grid_arrays(*grid)
    prm = drift_params(gaussian_params(n, seed, k_max), step)
    idx = np.arange(n) if idx is None else np.asarray(idx)
    x = _eval_numpy(prm, idx, vpar, vperp).reshape(len(idx), grid[0] * grid[1])
    if heavy_frac > 0.0:
        x = _add_heavy_tail_numpy(x, n, seed, heavy_frac, idx)
    return np.ascontiguousarray(x)


def _heavy_rows(n: int, seed: int, heavy_frac: float):
    rng = np.random.Generator(np.random.Philox(seed + 7919))
    return rng.random(n) < heavy_frac


def _add_heavy_tail_numpy(x, n, seed, heavy_frac, idx):
    heavy = _heavy_rows(n, seed, heavy_frac)
    for r, b in enumerate(idx):
        if heavy[b]:
            rng = np.random.Generator(np.random.Philox([seed + 104729, int(b)]))
            t = np.abs(rng.standard_t(2.0, size=x.shape[1]))
            x[r] += 1e-6 * x[r].max() * np.minimum(t, 1e3)
    return x


def histograms_torch(n: int, seed: int, device, k_max: int = 3, heavy_frac: float = 0.0,
                     chunk: int = 1 << 17, step: int = 0, grid=(N_PAR, N_PERP), rows=None):
    """Same workload as :func:`histograms` evaluated on a torch device in chunks
    (values may differ from the numpy evaluation in the last ulp; the device
    copy is what both sides of a comparison consume).  ``rows`` selects rows
    of the n-histogram workload (same values as the full set at those rows;
    without a heavy tail)."""
    import torch
    vpar, vperp, _ = grid_arrays(*grid)
    Pg = grid[0] * grid[1]
    prm = drift_params(gaussian_params(n, seed, k_max), step)
    if rows is not None:
        if heavy_frac > 0.0:
            raise ValueError("histograms_torch: rows= with a heavy tail is not supported")
        rows = np.asarray(rows, dtype=np.int64)
        prm = {k: v[rows] for k, v in prm.items()}
        n = len(rows)
    tv = torch.as_tensor(vpar, device=device)
    tq = torch.as_tensor(vperp, device=device)
    out = torch.empty((n, Pg), dtype=torch.float64, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        a = {k: torch.as_tensor(v[s:e], device=device) for k, v in prm.items()}
        ea = torch.exp(-(tv[None, None, :] - a["c_par"][:, :, None]) ** 2
                       / (2.0 * a["s_par"][:, :, None] ** 2))
        eb = torch.exp(-(tq[None, None, :] - a["c_perp"][:, :, None]) ** 2
                       / (2.0 * a["s_perp"][:, :, None] ** 2))
        x = torch.einsum("nk,nki,nkj->nji", a["amp"], ea, eb) * tq[None, :, None]
        out[s:e] = x.reshape(e - s, Pg)
    if heavy_frac > 0.0:
        heavy = np.nonzero(_heavy_rows(n, seed, heavy_frac))[0]
        g = torch.Generator(device=device)
        g.manual_seed(seed + 104729)
        for s in range(0, len(heavy), chunk):
            rows = torch.as_tensor(heavy[s:s + chunk], device=device)
            z = torch.randn((len(rows), Pg), generator=g, device=device, dtype=torch.float64)
            u = torch.rand((len(rows), Pg), generator=g, device=device, dtype=torch.float64)
            t = (z / torch.sqrt(-torch.log1p(-u))).abs().clamp_max(1e3)
            mx = out[rows].amax(dim=1, keepdim=True)
            out[rows] += 1e-6 * mx * t
    return out


def stand_in_xhat(x: np.ndarray, seed: int, rel: float = 1e-2, floor: float = 2e-3,
                  ld: int = 1536) -> np.ndarray:
    """A stand-in for a decoded histogram: x plus relative and absolute noise,
    rounded to float32, in rows of ``ld`` floats (padding zero)."""
    rng = np.random.Generator(np.random.Philox(seed + 31337))
    n, p = x.shape
    mx = x.max(axis=1, keepdims=True)
    noisy = x * (1.0 + rel * rng.standard_normal((n, p))) + floor * mx * rng.standard_normal((n, p))
    out = np.zeros((n, ld), np.float32)
    out[:, :p] = noisy.astype(np.float32)
    return out


def group_sizes(n_groups: int, seed: int, median: float = 8192.0, sigma_ln: float = 0.85,
                lo: int = 1024, hi: int = 65536) -> np.ndarray:
    rng = np.random.Generator(np.random.Philox(seed + 4242))
    g = np.exp(np.log(median) + sigma_ln * rng.standard_normal(n_groups))
    return np.clip(np.rint(g), lo, hi).astype(np.int64)


def ae_init(P: int, H: int, L: int, seed: int, tied: bool = True):
    """Fan-in uniform init U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for the dense
    layers (weights [in][out]), zero biases, identity normalisation."""
    rng = np.random.Generator(np.random.Philox(seed + 99991))
    W1 = rng.uniform(-1, 1, size=(P, H)) / np.sqrt(P)
    W2 = rng.uniform(-1, 1, size=(H, L)) / np.sqrt(H)
    d = dict(W1=W1, b1=np.zeros(H), W2=W2, b2=np.zeros(L), b3=np.zeros(H), b4=np.zeros(P),
             mu=np.zeros(P), sigma=np.ones(P))
    if not tied:
        d["W3"] = rng.uniform(-1, 1, size=(L, H)) / np.sqrt(L)
        d["W4"] = rng.uniform(-1, 1, size=(H, P)) / np.sqrt(H)
    return d


def mlp_init(nin: int, nh: int, nout: int, seed: int):
    rng = np.random.Generator(np.random.Philox(seed + 77777))
    return dict(W1=rng.uniform(-1, 1, size=(nin, nh)) * np.sqrt(6.0 / nin),
                b1=np.zeros(nh),
                W2=rng.uniform(-1, 1, size=(nh, nh)) * np.sqrt(6.0 / nh),
                b2=np.zeros(nh),
                W3=rng.uniform(-1, 1, size=(nh, nout)) / np.sqrt(nh),
                b3=np.zeros(nout))
