"""FP64 CPU oracle for the hybrid compressor's hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import this package.  It wraps ``aeqc_oracle.c`` (plain C, FP64,
plain loops) with ctypes and numpy.  It shares no code with the CUDA library.

Parity pins: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, brute force, finite differences,
exact rational arithmetic); see ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aeqc_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# status bits (same meaning as the library's; defined here independently)
CONVERGED = 0x0001
ROUND2 = 0x0002
VERBATIM = 0x0004
NONFINITE_INPUT = 0x0008
ZERO_IMAGE = 0x0010
CODE_ESCAPE = 0x0020
WARM_REJECTED = 0x0040
ALPHA_RETRY = 0x0080
AE_EXACT = 0x0100
ESCAPE = -32768
ZERO_CODE = -32767
CODE_MAX = 32766


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so with gcc (OpenMP if present)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
            "-o", _SO + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class _Grid(C.Structure):
    _fields_ = [("n_par", C.c_int), ("n_perp", C.c_int),
                ("vpar", C.c_void_p), ("vperp", C.c_void_p), ("vol", C.c_void_p),
                ("vol_uniform", C.c_double), ("mass", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("tau", C.c_double), ("alpha", C.c_double), ("step_s", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int), ("r2_max_iter", C.c_int),
                ("loss", C.c_int), ("warm_iters", C.c_int),
                ("warm_reject", C.c_double), ("qoi_check", C.c_double)]


class _AE(C.Structure):
    _fields_ = [("P", C.c_int), ("H", C.c_int), ("L", C.c_int), ("tied", C.c_int),
                ("act", C.c_int)] + [(nm, C.c_void_p) for nm in
                                     ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4",
                                      "mu", "sigma")]


class _MLP(C.Structure):
    _fields_ = [("nin", C.c_int), ("nh", C.c_int), ("nout", C.c_int)] + [
        (nm, C.c_void_p) for nm in ("W1", "b1", "W2", "b2", "W3", "b3",
                                    "in_mu", "in_sd", "out_mu", "out_sd")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
            sig = {
                "or_moments": [vp, vp, i64, vp],
                "or_abs_moments": [vp, vp, i64, vp],
                "or_qois_from_moments": [vp, i64, dbl, vp],
                "or_qois_direct": [vp, vp, i64, vp],
                "or_delta": [dbl, dbl],
                "or_round_residual": [dbl, dbl, dbl],
                "or_quantize": [vp, vp, i64, i64, i32, dbl, dbl, vp, vp, vp, vp, vp],
                "or_dequantize": [vp, i64, vp, vp, vp, i64, i32, vp],
                "or_cholesky_solve4": [vp, vp, vp],
                "or_newton": [vp, vp, vp, i64, vp, i32, vp, vp, vp, vp],
                "or_newton_round1": [vp, vp, vp, i64, vp, vp, vp, vp],
                "or_compress_correct": [vp, vp, vp, i64, i64, vp, vp, vp, vp, vp, vp,
                                        vp, vp],
                "or_decompress": [vp, vp, i64, vp, vp, vp, vp, vp, i64, vp, vp],
                "or_nrmse": [vp, vp, i64],
                "or_ae_forward": [vp, vp, i64, vp, vp, vp],
                "or_ae_decode": [vp, vp, vp, i64, vp],
                "or_ae_loss_grad": [vp, vp, i64] + [vp] * 8,
                "or_adam": [vp, vp, vp, vp, i64, dbl, dbl, dbl, dbl, i32],
                "or_fit_normalizer": [vp, i64, i32, dbl, vp, vp],
                "or_mlp_predict": [vp, vp, i64, vp],
                "or_mlp_loss_grad": [vp, vp, vp, i64] + [vp] * 6,
                "or_num_threads": [],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = None
            for name in ("or_delta", "or_round_residual", "or_nrmse",
                         "or_ae_loss_grad", "or_mlp_loss_grad"):
                getattr(L, name).restype = C.c_double
            L.or_cholesky_solve4.restype = C.c_int
            L.or_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Grid:
    """Velocity grid: v_par (index i, fastest), v_perp (index j), cell volumes."""
    vpar: np.ndarray
    vperp: np.ndarray
    vol_uniform: float
    vol: Optional[np.ndarray] = None
    mass: float = 1.0

    def __post_init__(self):
        self.vpar = _f64(self.vpar)
        self.vperp = _f64(self.vperp)
        if self.vol is not None:
            self.vol = _f64(self.vol)

    @property
    def P(self) -> int:
        return len(self.vpar) * len(self.vperp)

    def c(self) -> _Grid:
        return _Grid(len(self.vpar), len(self.vperp), _p(self.vpar), _p(self.vperp),
                     _p(self.vol), float(self.vol_uniform), float(self.mass))


@dataclass
class Params:
    tau: float = 1e-4
    alpha: float = 0.5
    step_s: float = 1.0
    tol: float = 1e-12
    max_iter: int = 50
    r2_max_iter: int = 400
    loss: int = 0
    warm_iters: int = 2
    warm_reject: float = 1e-8
    qoi_check: float = 1e-10

    def c(self) -> _Params:
        return _Params(self.tau, self.alpha, self.step_s, self.tol, self.max_iter,
                       self.r2_max_iter, self.loss, self.warm_iters, self.warm_reject,
                       self.qoi_check)


def num_threads() -> int:
    return int(lib().or_num_threads())


# --- Eq. (1)-(4) -------------------------------------------------------------

def moments(grid: Grid, x) -> np.ndarray:
    x = _f64(x).reshape(-1, grid.P)
    Q = np.zeros((x.shape[0], 4))
    g = grid.c()
    lib().or_moments(C.byref(g), _p(x), x.shape[0], _p(Q))
    return Q


def abs_moments(grid: Grid, x) -> np.ndarray:
    x = _f64(x).reshape(-1, grid.P)
    S = np.zeros((x.shape[0], 4))
    g = grid.c()
    lib().or_abs_moments(C.byref(g), _p(x), x.shape[0], _p(S))
    return S


def qois_from_moments(Q, mass: float = 1.0) -> np.ndarray:
    Q = _f64(Q).reshape(-1, 4)
    out = np.zeros_like(Q)
    lib().or_qois_from_moments(_p(Q), Q.shape[0], float(mass), _p(out))
    return out


def qois_direct(grid: Grid, x) -> np.ndarray:
    x = _f64(x).reshape(-1, grid.P)
    out = np.zeros((x.shape[0], 4))
    g = grid.c()
    lib().or_qois_direct(C.byref(g), _p(x), x.shape[0], _p(out))
    return out


# --- Stage 4: quantizer -----------------------------------------------------

def delta(e: float, alpha: float) -> float:
    return float(lib().or_delta(float(e), float(alpha)))


def round_residual(x: float, xh: float, dl: float) -> float:
    return float(lib().or_round_residual(float(x), float(xh), float(dl)))


def _xhat2d(xhat, n, P):
    xhat = np.ascontiguousarray(xhat, dtype=np.float32)
    if xhat.ndim == 1:
        xhat = xhat.reshape(n, -1)
    xhat = xhat.reshape(n, -1)
    assert xhat.shape[1] >= P
    return xhat


def quantize(x, xhat, tau: float, alpha: float = 0.5):
    """Codes int16 [n][P], x' [n][P], scale [n], delta [n], status [n]."""
    x = _f64(x)
    n = x.shape[0]
    P = x.reshape(n, -1).shape[1]
    x = x.reshape(n, P)
    xhat = _xhat2d(xhat, n, P)
    codes = np.zeros((n, P), np.int16)
    xp = np.zeros((n, P))
    scale = np.zeros(n)
    dl = np.zeros(n)
    st = np.zeros(n, np.uint16)
    lib().or_quantize(_p(x), _p(xhat), xhat.shape[1], n, P, float(tau), float(alpha),
                      _p(codes), _p(xp), _p(scale), _p(dl), _p(st))
    return codes, xp, scale, dl, st


def dequantize(xhat, codes, raw, dl) -> np.ndarray:
    codes = np.ascontiguousarray(codes, np.int16)
    n, P = codes.shape
    xhat = _xhat2d(xhat, n, P)
    raw = _f64(raw).reshape(n, P)
    dl = _f64(dl)
    out = np.zeros((n, P))
    lib().or_dequantize(_p(xhat), xhat.shape[1], _p(codes), _p(raw), _p(dl), n, P, _p(out))
    return out


# --- Stage 5: Newton --------------------------------------------------------

def newton(grid: Grid, xprime, Q, params: Params = None, lam0=None):
    """Solve for lambda; returns lam [n][4], f [n][P], iters [n], status [n]."""
    params = params or Params()
    xp = _f64(xprime).reshape(-1, grid.P)
    n = xp.shape[0]
    Q = _f64(Q).reshape(n, 4)
    lam = np.zeros((n, 4)) if lam0 is None else _f64(lam0).reshape(n, 4).copy()
    f = np.zeros((n, grid.P))
    it = np.zeros(n, np.int32)
    st = np.zeros(n, np.uint16)
    g, pr = grid.c(), params.c()
    lib().or_newton(C.byref(g), _p(xp), _p(Q), n, C.byref(pr), int(lam0 is not None),
                    _p(lam), _p(f), _p(it), _p(st))
    return lam, f, it, st


def newton_round1(grid: Grid, xprime, Q, params: Params, lam0=None):
    """Round 1 only: plain Newton steps from lam0 (default 0); lam, iters, conv."""
    xp = _f64(xprime).reshape(-1, grid.P)
    n = xp.shape[0]
    Q = _f64(Q).reshape(n, 4)
    lam = np.zeros((n, 4)) if lam0 is None else _f64(lam0).reshape(n, 4).copy()
    it = np.zeros(n, np.int32)
    conv = np.zeros(n, np.int32)
    g, pr = grid.c(), params.c()
    lib().or_newton_round1(C.byref(g), _p(xp), _p(Q), n, C.byref(pr), _p(lam), _p(it),
                           _p(conv))
    return lam, it, conv


def cholesky_solve4(M, r):
    M = _f64(M).reshape(16)
    r = _f64(r).reshape(4)
    d = np.zeros(4)
    rc = lib().or_cholesky_solve4(_p(M), _p(r), _p(d))
    return rc, d


def compress_correct(grid: Grid, x, xhat, params: Params = None, lam0=None):
    """Stages 4+5 for a batch given xhat: codes, lam, scale, iters, status, f."""
    params = params or Params()
    x = _f64(x).reshape(-1, grid.P)
    n = x.shape[0]
    xhat = _xhat2d(xhat, n, grid.P)
    codes = np.zeros((n, grid.P), np.int16)
    lam = np.zeros((n, 4))
    scale = np.zeros(n)
    it = np.zeros(n, np.int32)
    st = np.zeros(n, np.uint16)
    f = np.zeros((n, grid.P))
    l0 = None if lam0 is None else _f64(lam0).reshape(n, 4)
    g, pr = grid.c(), params.c()
    lib().or_compress_correct(C.byref(g), _p(x), _p(xhat), xhat.shape[1], n, C.byref(pr),
                              _p(l0), _p(codes), _p(lam), _p(scale), _p(it), _p(st), _p(f))
    return dict(codes=codes, lam=lam, scale=scale, iters=it, status=st, f=f)


def decompress(grid: Grid, xhat, codes, raw, scale, lam, status, params: Params = None):
    params = params or Params()
    codes = np.ascontiguousarray(codes, np.int16).reshape(-1, grid.P)
    n = codes.shape[0]
    xhat = _xhat2d(xhat, n, grid.P)
    raw = _f64(raw).reshape(n, grid.P)
    scale, lam = _f64(scale), _f64(lam).reshape(n, 4)
    status = np.ascontiguousarray(status, np.uint16)
    f = np.zeros((n, grid.P))
    g, pr = grid.c(), params.c()
    lib().or_decompress(C.byref(g), _p(xhat), xhat.shape[1], _p(codes), _p(raw), _p(scale),
                        _p(lam), _p(status), n, C.byref(pr), _p(f))
    return f


# --- Eq. (7) ----------------------------------------------------------------

def nrmse(u, f) -> float:
    u, f = _f64(u).ravel(), _f64(f).ravel()
    return float(lib().or_nrmse(_p(u), _p(f), u.size))


# --- Autoencoder ------------------------------------------------------------

@dataclass
class AE:
    """FP64 autoencoder parameters; W stored [in][out]."""
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    b3: np.ndarray
    b4: np.ndarray
    mu: np.ndarray
    sigma: np.ndarray
    W3: Optional[np.ndarray] = None
    W4: Optional[np.ndarray] = None
    act: int = 0
    _keep: list = field(default_factory=list, repr=False)

    def __post_init__(self):
        for nm in ("W1", "b1", "W2", "b2", "b3", "b4", "mu", "sigma", "W3", "W4"):
            v = getattr(self, nm)
            if v is not None:
                setattr(self, nm, _f64(v))

    @property
    def tied(self) -> bool:
        return self.W3 is None

    def c(self) -> _AE:
        P, H = self.W1.shape
        L = self.W2.shape[1]
        return _AE(P, H, L, int(self.tied), int(self.act), _p(self.W1), _p(self.b1),
                   _p(self.W2), _p(self.b2), _p(self.W3), _p(self.b3), _p(self.W4),
                   _p(self.b4), _p(self.mu), _p(self.sigma))


def ae_forward(m: AE, x):
    P, H = m.W1.shape
    L = m.W2.shape[1]
    x = _f64(x).reshape(-1, P)
    n = x.shape[0]
    z = np.zeros((n, L))
    xh = np.zeros((n, P))
    s = np.zeros(n)
    mc = m.c()
    lib().or_ae_forward(C.byref(mc), _p(x), n, _p(z), _p(xh), _p(s))
    return z, xh, s


def ae_decode(m: AE, z, scale):
    P = m.W1.shape[0]
    z = _f64(z)
    n = z.shape[0]
    scale = _f64(scale)
    xh = np.zeros((n, P))
    mc = m.c()
    lib().or_ae_decode(C.byref(mc), _p(z), _p(scale), n, _p(xh))
    return xh


def ae_loss_grad(m: AE, x):
    P, H = m.W1.shape
    L = m.W2.shape[1]
    x = _f64(x).reshape(-1, P)
    g = dict(W1=np.zeros((P, H)), b1=np.zeros(H), W2=np.zeros((H, L)), b2=np.zeros(L),
             W3=np.zeros((L, H)), b3=np.zeros(H), W4=np.zeros((H, P)), b4=np.zeros(P))
    mc = m.c()
    loss = lib().or_ae_loss_grad(C.byref(mc), _p(x), x.shape[0], _p(g["W1"]), _p(g["b1"]),
                                 _p(g["W2"]), _p(g["b2"]), _p(g["W3"]), _p(g["b3"]),
                                 _p(g["W4"]), _p(g["b4"]))
    if m.tied:
        g.pop("W3"), g.pop("W4")
    return float(loss), g


def adam(w, grad, m1, m2, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, t=1):
    """In-place Adam update of float64 arrays w, m1, m2."""
    for a in (w, m1, m2):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    grad = _f64(grad)
    lib().or_adam(_p(w), _p(grad), _p(m1), _p(m2), w.size, lr, beta1, beta2, eps, int(t))


def fit_normalizer(x, P: int, floor_sigma: float = 1e-6):
    x = _f64(x).reshape(-1, P)
    mu, sd = np.zeros(P), np.zeros(P)
    lib().or_fit_normalizer(_p(x), x.shape[0], P, floor_sigma, _p(mu), _p(sd))
    return mu, sd


# --- Warm-start MLP -----------------------------------------------------------

@dataclass
class MLP:
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray
    in_mu: np.ndarray
    in_sd: np.ndarray
    out_mu: np.ndarray
    out_sd: np.ndarray

    def __post_init__(self):
        for nm in ("W1", "b1", "W2", "b2", "W3", "b3", "in_mu", "in_sd", "out_mu", "out_sd"):
            setattr(self, nm, _f64(getattr(self, nm)))

    def c(self) -> _MLP:
        nin, nh = self.W1.shape
        nout = self.W3.shape[1]
        return _MLP(nin, nh, nout, *[_p(getattr(self, nm)) for nm in
                                     ("W1", "b1", "W2", "b2", "W3", "b3", "in_mu",
                                      "in_sd", "out_mu", "out_sd")])


def mlp_predict(m: MLP, inp):
    nin = m.W1.shape[0]
    inp = _f64(inp).reshape(-1, nin)
    out = np.zeros((inp.shape[0], m.W3.shape[1]))
    mc = m.c()
    lib().or_mlp_predict(C.byref(mc), _p(inp), inp.shape[0], _p(out))
    return out


def mlp_loss_grad(m: MLP, inp, target):
    nin, nh = m.W1.shape
    no = m.W3.shape[1]
    inp = _f64(inp).reshape(-1, nin)
    target = _f64(target).reshape(-1, no)
    g = dict(W1=np.zeros((nin, nh)), b1=np.zeros(nh), W2=np.zeros((nh, nh)), b2=np.zeros(nh),
             W3=np.zeros((nh, no)), b3=np.zeros(no))
    mc = m.c()
    loss = lib().or_mlp_loss_grad(C.byref(mc), _p(inp), _p(target), inp.shape[0],
                                  *[_p(g[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    return float(loss), g
