"""Thin Python binding of libaeqc (ctypes).

Argument marshalling only: torch tensors become raw device pointers and the
current CUDA stream; every step of the hot path runs in the library's own
CUDA kernels.  Loading fails loudly when the library is missing -- there is
no CPU fallback.

Names follow the C ABI in ``include/aeqc.h``.
"""
from __future__ import annotations

import ctypes as C
import struct
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaeqc.so")

OK, EINVAL, ECUDA, ENOMEM, ECORRUPT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5
ST_CONVERGED = 0x0001
ST_ROUND2 = 0x0002
ST_VERBATIM = 0x0004
ST_NONFINITE_INPUT = 0x0008
ST_ZERO_IMAGE = 0x0010
ST_CODE_ESCAPE = 0x0020
ST_WARM_REJECTED = 0x0040
ST_ALPHA_RETRY = 0x0080
ST_AE_EXACT = 0x0100
ST_OUTLIER_OVERFLOW = 0x0200
CODE_ESCAPE = -32768
CODE_ZERO = -32767
CODE_MAX = 32766
XHAT_LD = 1536
KERNEL_FP64 = 0
KERNEL_FAST = 1
DTYPE_F32 = 0
DTYPE_BF16 = 1
ACT_IDENTITY = 0
ACT_RELU = 1


class AeqcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"aeqc error {code}: {msg}")
        self.code = code


# --- structs (mirror include/aeqc.h) ---------------------------------------

class aeqc_grid(C.Structure):
    _fields_ = [("n_par", C.c_int32), ("n_perp", C.c_int32), ("vpar_host", C.c_void_p),
                ("vperp_host", C.c_void_p), ("vol", C.c_void_p), ("vol_uniform", C.c_double),
                ("mass", C.c_double)]


class aeqc_params(C.Structure):
    _fields_ = [("tau", C.c_double), ("alpha", C.c_double), ("step_s", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int32), ("r2_max_iter", C.c_int32),
                ("loss", C.c_int32), ("warm_iters", C.c_int32), ("warm_reject", C.c_double),
                ("qoi_check", C.c_double), ("kernel", C.c_int32), ("reserved", C.c_int32)]


class aeqc_model_desc(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("P", "H", "L", "tied", "act", "dtype", "n_groups",
                                          "layers")]


class aeqc_tuning(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("enc_stages", "dec_stages", "qc_warps_per_sm",
                                          "reserved")]


class aeqc_outliers(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("count", C.c_void_p), ("index", C.c_void_p),
                ("value", C.c_void_p)]


class aeqc_compressed(C.Structure):
    _fields_ = [("latent", C.c_void_p), ("scale", C.c_void_p), ("codes", C.c_void_p),
                ("lambda_", C.c_void_p), ("iters", C.c_void_p), ("status", C.c_void_p),
                ("outliers", aeqc_outliers), ("features", C.c_void_p)]


_lib = None
SYMBOLS = {
    "aeqc_params_default": (None, [C.c_void_p]),
    "aeqc_last_error": (C.c_char_p, []),
    "aeqc_version": (C.c_char_p, []),
    "aeqc_model_create": (C.c_int, [C.c_void_p, C.c_void_p]),
    "aeqc_model_destroy": (C.c_int, [C.c_void_p]),
    "aeqc_model_set_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "aeqc_model_get_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "aeqc_model_device_status": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "aeqc_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                C.c_void_p, C.c_void_p]),
    "aeqc_model_set_group": (C.c_int, [C.c_void_p, C.c_int32] + [C.c_void_p] * 10),
    "aeqc_model_get_group": (C.c_int, [C.c_void_p, C.c_int32] + [C.c_void_p] * 10),
    "aeqc_fit_normalizer": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64,
                                      C.c_void_p, C.c_size_t, C.c_void_p]),
    "aeqc_fit_normalizer_workspace_size": (C.c_size_t, [C.c_void_p]),
    "ae_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_float,
                                C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ae_train_workspace_size": (C.c_size_t, [C.c_void_p, C.c_int64]),
    "aeqc_model_param_count": (C.c_int64, [C.c_void_p]),
    "ae_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ae_encode": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ae_encode_workspace_size": (C.c_size_t, [C.c_void_p, C.c_int64]),
    "ae_decode": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                            C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ae_decode_workspace_size": (C.c_size_t, [C.c_void_p, C.c_int64]),
    "residual_quantize": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "residual_dequantize": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
    "qoi_moments": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "qoi_correct": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                              C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p]),
    "compress_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                 C.c_void_p]),
    "compress_batch_workspace_size": (C.c_size_t, [C.c_void_p, C.c_int64]),
    "compress_batch_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_int64, C.c_void_p, C.c_void_p, C.c_int64,
                                      C.c_void_p, C.c_size_t, C.c_void_p]),
    "compress_batch_host_workspace_size": (C.c_size_t, [C.c_void_p, C.c_int64, C.c_int64]),
    "quantize_correct": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                                   C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "quantize_correct_workspace_size": (C.c_size_t, [C.c_int64]),
    "quantize_correct_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                           C.c_int64, C.c_void_p, C.c_void_p, C.c_int32,
                                           C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "decompress_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                   C.c_void_p]),
    "decompress_batch_workspace_size": (C.c_size_t, [C.c_void_p, C.c_int64]),
    "aeqc_mlp_create": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p]),
    "aeqc_mlp_destroy": (C.c_int, [C.c_void_p]),
    "aeqc_mlp_set": (C.c_int, [C.c_void_p] + [C.c_void_p] * 10),
    "aeqc_mlp_get": (C.c_int, [C.c_void_p] + [C.c_void_p] * 6),
    "mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                                 C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "mlp_train_workspace_size": (C.c_size_t, [C.c_void_p, C.c_int64]),
    "aeqc_mlp_param_count": (C.c_int64, [C.c_void_p]),
    "mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "mlp_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "pq_train_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32]),
    "pq_train": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_int32,
                           C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_size_t,
                           C.c_void_p]),
    "pq_encode": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_int32,
                            C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pq_decode": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                            C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "rice_workspace_size": (C.c_size_t, [C.c_int64]),
    "rice_measure": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "rice_pack": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_int64, C.c_void_p]),
    "rice_unpack": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64,
                              C.c_int32, C.c_void_p, C.c_void_p]),
    "nrmse_workspace_size": (C.c_size_t, [C.c_int64]),
    "nrmse_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "aeqc_bound_search_workspace_size": (C.c_size_t, [C.c_void_p, C.c_int64, C.c_int64]),
    "aeqc_bound_search": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                    C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int32,
                                    C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                    C.c_void_p]),
    "aeqc_model_save_size": (C.c_size_t, [C.c_void_p]),
    "aeqc_model_save": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "aeqc_model_load": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p]),
    "aeqc_mlp_save_size": (C.c_size_t, [C.c_void_p]),
    "aeqc_mlp_save": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "aeqc_mlp_load": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p]),
    "aeqc_batch_pack_size": (C.c_size_t, [C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                          C.c_int64]),
    "aeqc_batch_pack": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                  C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "aeqc_batch_peek": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "aeqc_batch_unpack": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "aeqc_partition_lpt": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                     C.c_void_p]),
    "aeqc_exclusive_scan": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
}


def load(path: str = LIB_PATH):
    """Load libaeqc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libaeqc.so not built ({path}); run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (res, args) in SYMBOLS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise AeqcError(rc, load().aeqc_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream=None) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _workspace(nbytes: int, device):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def params_default(**kw) -> aeqc_params:
    p = aeqc_params()
    load().aeqc_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Grid:
    """Velocity grid (host v_par / v_perp arrays; device vol or uniform)."""

    def __init__(self, vpar, vperp, vol_uniform: float, vol=None, mass: float = 1.0):
        self.vpar = np.ascontiguousarray(vpar, np.float64)
        self.vperp = np.ascontiguousarray(vperp, np.float64)
        self.vol = vol
        self.c = aeqc_grid(len(self.vpar), len(self.vperp), self.vpar.ctypes.data,
                           self.vperp.ctypes.data, _ptr(vol), float(vol_uniform), float(mass))

    @property
    def P(self) -> int:
        return len(self.vpar) * len(self.vperp)


# --- residual quantizer / correction --------------------------------------

def residual_quantize(x, xhat, params: aeqc_params, outlier_capacity: int = 0,
                      want_xrec: bool = False, stream=None):
    import torch
    n, P = x.shape
    dev = x.device
    codes = torch.empty((n, P), dtype=torch.int16, device=dev)
    scale = torch.empty(n, dtype=torch.float64, device=dev)
    status = torch.empty(n, dtype=torch.uint16, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    idx = torch.empty(max(outlier_capacity, 1), dtype=torch.int64, device=dev)
    val = torch.empty(max(outlier_capacity, 1), dtype=torch.float64, device=dev)
    out = aeqc_outliers(outlier_capacity, _ptr(cnt), _ptr(idx), _ptr(val))
    xrec = torch.empty((n, P), dtype=torch.float64, device=dev) if want_xrec else None
    _check(load().residual_quantize(_ptr(x), _ptr(xhat), xhat.stride(0), n, P,
                                    C.byref(params), _ptr(codes), _ptr(scale), _ptr(status),
                                    C.byref(out), _ptr(xrec), _stream(stream)))
    return dict(codes=codes, scale=scale, status=status, count=cnt, index=idx, value=val,
                xrec=xrec, outliers=out)


def residual_dequantize(xhat, codes, scale, status, params: aeqc_params, outliers=None,
                        stream=None):
    import torch
    n, P = codes.shape
    xrec = torch.empty((n, P), dtype=torch.float64, device=codes.device)
    _check(load().residual_dequantize(_ptr(xhat), xhat.stride(0), _ptr(codes),
                                      C.byref(outliers) if outliers is not None else None,
                                      _ptr(scale), _ptr(status), n, P, C.byref(params),
                                      _ptr(xrec), _stream(stream)))
    return xrec


def qoi_moments(grid: Grid, x, stream=None):
    import torch
    Q = torch.empty((x.shape[0], 4), dtype=torch.float64, device=x.device)
    _check(load().qoi_moments(C.byref(grid.c), _ptr(x), x.shape[0], _ptr(Q), _stream(stream)))
    return Q


def qoi_correct(grid: Grid, xrec, Q, params: aeqc_params, lam0=None, want_f: bool = False,
                stream=None):
    import torch
    n = xrec.shape[0]
    dev = xrec.device
    lam = lam0.clone() if lam0 is not None else torch.zeros((n, 4), dtype=torch.float64,
                                                             device=dev)
    f = torch.empty_like(xrec) if want_f else None
    iters = torch.empty(n, dtype=torch.uint8, device=dev)
    status = torch.empty(n, dtype=torch.uint16, device=dev)
    _check(load().qoi_correct(C.byref(grid.c), _ptr(xrec), _ptr(Q), n, C.byref(params),
                              int(lam0 is not None), _ptr(lam), _ptr(f), _ptr(iters),
                              _ptr(status), _stream(stream)))
    return dict(lam=lam, f=f, iters=iters, status=status)


# --- autoencoder ------------------------------------------------------------

class Model:
    """Autoencoder handle (aeqc_model)."""

    def __init__(self, P: int, H: int, L: int, tied: bool = True, act: int = ACT_IDENTITY,
                 dtype: int = DTYPE_F32, n_groups: int = 1, layers: int = 2):
        """layers = 1: the paper's single tied linear layer P -> L -> P (H must be L)."""
        self.desc = aeqc_model_desc(P, H, L, int(tied), act, dtype, n_groups, layers)
        self.h = C.c_void_p()
        _check(load().aeqc_model_create(C.byref(self.desc), C.byref(self.h)))

    def close(self):
        if self.h:
            load().aeqc_model_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self) -> bytes:
        """Checkpoint blob (weights, normalisation, Adam state, steps)."""
        lib = load()
        buf = C.create_string_buffer(lib.aeqc_model_save_size(self.h))
        _check(lib.aeqc_model_save(self.h, buf, len(buf)))
        return buf.raw

    @classmethod
    def load(cls, blob: bytes) -> "Model":
        """Model restored from a save() blob (AeqcError ECORRUPT if invalid)."""
        self = cls.__new__(cls)
        self.h = C.c_void_p()
        _check(load().aeqc_model_load(blob, len(blob), C.byref(self.h)))
        self.desc = aeqc_model_desc.from_buffer_copy(blob[16:16 + C.sizeof(aeqc_model_desc)])
        return self

    @property
    def P(self):
        return self.desc.P

    @property
    def H(self):
        return self.desc.H

    @property
    def L(self):
        return self.desc.L

    def set_group(self, g: int, p: dict):
        f = lambda k: (np.ascontiguousarray(p[k], np.float64) if p.get(k) is not None else None)
        arrs = [f(k) for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4", "mu", "sigma")]
        _check(load().aeqc_model_set_group(self.h, g, *[a.ctypes.data if a is not None else None
                                                        for a in arrs]))

    def get_group(self, g: int) -> dict:
        P, H, L = self.P, self.H, self.L
        tied = bool(self.desc.tied)
        out = dict(W1=np.zeros((P, H)), b1=np.zeros(H), W2=np.zeros((H, L)), b2=np.zeros(L),
                   W3=None if tied else np.zeros((L, H)), b3=np.zeros(H),
                   W4=None if tied else np.zeros((H, P)), b4=np.zeros(P), mu=np.zeros(P),
                   sigma=np.zeros(P))
        keys = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4", "mu", "sigma")
        _check(load().aeqc_model_get_group(self.h, g, *[out[k].ctypes.data if out[k] is not None
                                                         else None for k in keys]))
        return out

    def fit_normalizer(self, g: int, x, stream=None):
        ws = _workspace(8 * x.shape[0], x.device)
        _check(load().aeqc_fit_normalizer(self.h, g, _ptr(x), x.shape[0], _ptr(ws), ws.numel(),
                                          _stream(stream)))

    def train_step(self, x_batch, lr: float = 1e-3, group: int = 0, loss_out=None, ws=None,
                   stream=None):
        B = x_batch.shape[0]
        need = load().ae_train_workspace_size(self.h, B)
        if ws is None or ws.numel() < need:
            ws = _workspace(need, x_batch.device)
        _check(load().ae_train_step(self.h, _ptr(x_batch), B, group, lr, _ptr(loss_out),
                                    _ptr(ws), ws.numel(), _stream(stream)))
        return ws

    def loss_grad(self, x_batch, group: int = 0, stream=None):
        """(loss, flat FP32 gradient) of one batch without an update."""
        import torch
        B = x_batch.shape[0]
        ws = _workspace(load().ae_train_workspace_size(self.h, B), x_batch.device)
        g = torch.empty(load().aeqc_model_param_count(self.h), dtype=torch.float32,
                        device=x_batch.device)
        loss = torch.empty(1, dtype=torch.float32, device=x_batch.device)
        _check(load().ae_loss_grad(self.h, _ptr(x_batch), B, group, _ptr(loss), _ptr(g),
                                   _ptr(ws), ws.numel(), _stream(stream)))
        return loss, g

    def set_tuning(self, enc_stages: int = 0, dec_stages: int = 0, qc_warps_per_sm: int = 0):
        t = aeqc_tuning(enc_stages, dec_stages, qc_warps_per_sm, 0)
        _check(load().aeqc_model_set_tuning(self.h, C.byref(t)))

    def get_tuning(self) -> dict:
        t = aeqc_tuning()
        _check(load().aeqc_model_get_tuning(self.h, C.byref(t)))
        return dict(enc_stages=t.enc_stages, dec_stages=t.dec_stages,
                    qc_warps_per_sm=t.qc_warps_per_sm)

    def device_status(self, stream=None) -> int:
        """The model's device status word (nonzero: a bounded wait inside one
        of its tensor-core kernels ran out since the last read); read and
        cleared, synchronising the stream."""
        v = C.c_int32(0)
        _check(load().aeqc_model_device_status(self.h, C.byref(v), _stream(stream)))
        return v.value

    def latent_dtype(self):
        import torch
        return torch.bfloat16 if self.desc.dtype == DTYPE_BF16 else torch.float32


def ae_encode(m: Model, x, group_offsets=None, stream=None):
    import torch
    n = x.shape[0]
    latent = torch.empty((n, m.L), dtype=m.latent_dtype(), device=x.device)
    scale = torch.empty(n, dtype=torch.float64, device=x.device)
    ws = _workspace(load().ae_encode_workspace_size(m.h, n), x.device)
    _check(load().ae_encode(m.h, _ptr(x), n, _ptr(group_offsets), _ptr(latent), _ptr(scale),
                            _ptr(ws), ws.numel(), _stream(stream)))
    return latent, scale


def ae_decode(m: Model, latent, scale, group_offsets=None, ld: int = XHAT_LD, stream=None):
    import torch
    n = latent.shape[0]
    xhat = torch.empty((n, ld), dtype=torch.float32, device=latent.device)
    ws = _workspace(load().ae_decode_workspace_size(m.h, n), latent.device)
    _check(load().ae_decode(m.h, _ptr(latent), _ptr(scale), n, _ptr(group_offsets),
                            _ptr(xhat), ld, _ptr(ws), ws.numel(), _stream(stream)))
    return xhat


# --- warm-start MLP ---------------------------------------------------------

class MLP:
    def __init__(self, n_in: int, n_hidden: int = 64):
        self.n_in, self.nh = n_in, n_hidden
        self.h = C.c_void_p()
        _check(load().aeqc_mlp_create(n_in, n_hidden, C.byref(self.h)))

    def close(self):
        if self.h:
            load().aeqc_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self) -> bytes:
        """Checkpoint blob (weights, normalisation, Adam state, step)."""
        lib = load()
        buf = C.create_string_buffer(lib.aeqc_mlp_save_size(self.h))
        _check(lib.aeqc_mlp_save(self.h, buf, len(buf)))
        return buf.raw

    @classmethod
    def load(cls, blob: bytes) -> "MLP":
        """MLP restored from a save() blob (AeqcError ECORRUPT if invalid)."""
        self = cls.__new__(cls)
        self.h = C.c_void_p()
        _check(load().aeqc_mlp_load(blob, len(blob), C.byref(self.h)))
        self.n_in, self.nh = struct.unpack_from("<ii", blob, 16)
        return self

    def set(self, p: dict):
        keys = ("W1", "b1", "W2", "b2", "W3", "b3", "in_mu", "in_sd", "out_mu", "out_sd")
        arrs = [np.ascontiguousarray(p[k], np.float64) for k in keys]
        _check(load().aeqc_mlp_set(self.h, *[a.ctypes.data for a in arrs]))

    def get(self) -> dict:
        ni, nh = self.n_in, self.nh
        out = dict(W1=np.zeros((ni, nh)), b1=np.zeros(nh), W2=np.zeros((nh, nh)),
                   b2=np.zeros(nh), W3=np.zeros((nh, 4)), b3=np.zeros(4))
        _check(load().aeqc_mlp_get(self.h, *[out[k].ctypes.data for k in
                                             ("W1", "b1", "W2", "b2", "W3", "b3")]))
        return out

    def train_step(self, inputs, target_lambda, lr: float = 1e-3, loss_out=None, ws=None,
                   stream=None):
        B = inputs.shape[0]
        need = load().mlp_train_workspace_size(self.h, B)
        if ws is None or ws.numel() < need:
            ws = _workspace(need, inputs.device)
        _check(load().mlp_train_step(self.h, _ptr(inputs), _ptr(target_lambda), B, lr,
                                     _ptr(loss_out), _ptr(ws), ws.numel(), _stream(stream)))
        return ws

    def loss_grad(self, inputs, target_lambda, stream=None):
        import torch
        B = inputs.shape[0]
        ws = _workspace(load().mlp_train_workspace_size(self.h, B), inputs.device)
        g = torch.empty(load().aeqc_mlp_param_count(self.h), dtype=torch.float32,
                        device=inputs.device)
        loss = torch.empty(1, dtype=torch.float32, device=inputs.device)
        _check(load().mlp_loss_grad(self.h, _ptr(inputs), _ptr(target_lambda), B, _ptr(loss),
                                    _ptr(g), _ptr(ws), ws.numel(), _stream(stream)))
        return loss, g

    def predict(self, inputs, stream=None):
        import torch
        lam = torch.empty((inputs.shape[0], 4), dtype=torch.float64, device=inputs.device)
        _check(load().mlp_predict(self.h, _ptr(inputs), inputs.shape[0], _ptr(lam),
                                  _stream(stream)))
        return lam


# --- fused batch calls --------------------------------------------------------

class Compressed:
    """Device buffers of a compressed batch (aeqc_compressed)."""

    def __init__(self, n: int, P: int, L: int, latent_dtype, device, outlier_capacity: int,
                 features: bool = False):
        import torch
        self.n = n
        self.latent = torch.empty((n, L), dtype=latent_dtype, device=device)
        self.scale = torch.empty(n, dtype=torch.float64, device=device)
        self.codes = torch.empty((n, P), dtype=torch.int16, device=device)
        self.lam = torch.empty((n, 4), dtype=torch.float64, device=device)
        self.iters = torch.empty(n, dtype=torch.uint8, device=device)
        self.status = torch.empty(n, dtype=torch.uint16, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        cap = max(int(outlier_capacity), 1)
        self.index = torch.empty(cap, dtype=torch.int64, device=device)
        self.value = torch.empty(cap, dtype=torch.float64, device=device)
        self.features = (torch.empty((n, L + 4), dtype=torch.float32, device=device)
                         if features else None)
        self.c = aeqc_compressed(
            _ptr(self.latent), _ptr(self.scale), _ptr(self.codes), _ptr(self.lam),
            _ptr(self.iters), _ptr(self.status),
            aeqc_outliers(int(outlier_capacity), _ptr(self.count), _ptr(self.index),
                          _ptr(self.value)),
            _ptr(self.features))


class CompressedHost(Compressed):
    """Page-locked HOST buffers of a compressed batch (for compress_batch_host)."""

    def __init__(self, n: int, P: int, L: int, latent_dtype, outlier_capacity: int):
        import torch
        self.n = n
        pin = dict(device="cpu", pin_memory=True)
        self.latent = torch.empty((n, L), dtype=latent_dtype, **pin)
        self.scale = torch.empty(n, dtype=torch.float64, **pin)
        self.codes = torch.empty((n, P), dtype=torch.int16, **pin)
        self.lam = torch.empty((n, 4), dtype=torch.float64, **pin)
        self.iters = torch.empty(n, dtype=torch.uint8, **pin)
        self.status = torch.empty(n, dtype=torch.uint16, **pin)
        self.count = torch.zeros(1, dtype=torch.int64, **pin)
        cap = max(int(outlier_capacity), 1)
        self.index = torch.empty(cap, dtype=torch.int64, **pin)
        self.value = torch.empty(cap, dtype=torch.float64, **pin)
        self.features = None
        self.c = aeqc_compressed(
            _ptr(self.latent), _ptr(self.scale), _ptr(self.codes), _ptr(self.lam),
            _ptr(self.iters), _ptr(self.status),
            aeqc_outliers(int(outlier_capacity), _ptr(self.count), _ptr(self.index),
                          _ptr(self.value)),
            None)


def compress_batch_host(m: Model, grid: Grid, x_host, params: aeqc_params, chunk: int = 1 << 17,
                        mlp: Optional[MLP] = None, out: Optional[CompressedHost] = None,
                        ws=None, outlier_capacity: Optional[int] = None, device=None,
                        stream=None) -> CompressedHost:
    """compress_batch from a (page-locked) host array into host buffers, with
    the copies of one chunk overlapping the compute of the next."""
    import torch
    n, P = x_host.shape
    cap = outlier_capacity if outlier_capacity is not None else max(1024, 4 * n)
    if out is None:
        out = CompressedHost(n, P, m.L, m.latent_dtype(), cap)
    cap = out.c.outliers.capacity
    device = device or torch.device("cuda", torch.cuda.current_device())
    need = load().compress_batch_host_workspace_size(m.h, min(chunk, n), cap)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, device)
    _check(load().compress_batch_host(m.h, mlp.h if mlp is not None else None, C.byref(grid.c),
                                      _ptr(x_host), n, C.byref(params), C.byref(out.c), chunk,
                                      _ptr(ws), ws.numel(), _stream(stream)))
    out.ws = ws
    return out


def autotune(m: Model, grid: Grid, x, params: aeqc_params, mlp: Optional[MLP] = None,
             group_offsets=None, out: Optional[Compressed] = None, ws=None,
             outlier_capacity: Optional[int] = None, stream=None) -> dict:
    """Times the launch choices on this batch, keeps the fastest in the model
    and returns them (the outputs in `out` are those of compress_batch)."""
    n = x.shape[0]
    if out is None:
        cap = outlier_capacity if outlier_capacity is not None else max(1024, n * 4)
        out = Compressed(n, m.P, m.L, m.latent_dtype(), x.device, cap)
    if ws is None:
        ws = compress_batch_workspace(m, n, x.device)
    t = aeqc_tuning()
    _check(load().aeqc_autotune(m.h, mlp.h if mlp is not None else None, C.byref(grid.c),
                                _ptr(x), n, _ptr(group_offsets), C.byref(params),
                                C.byref(out.c), _ptr(ws), ws.numel(), _stream(stream),
                                C.byref(t)))
    return dict(enc_stages=t.enc_stages, dec_stages=t.dec_stages,
                qc_warps_per_sm=t.qc_warps_per_sm)


def compress_batch_workspace(m: Model, n: int, device):
    return _workspace(load().compress_batch_workspace_size(m.h, n), device)


def decompress_batch_workspace(m: Model, n: int, device):
    return _workspace(load().decompress_batch_workspace_size(m.h, n), device)


def compress_batch(m: Model, grid: Grid, x, params: aeqc_params, mlp: Optional[MLP] = None,
                   group_offsets=None, out: Optional[Compressed] = None, ws=None,
                   outlier_capacity: Optional[int] = None, features: bool = False,
                   stream=None) -> Compressed:
    n = x.shape[0]
    if out is None:
        cap = outlier_capacity if outlier_capacity is not None else max(1024, n * 4)
        out = Compressed(n, m.P, m.L, m.latent_dtype(), x.device, cap, features)
    if ws is None:
        ws = compress_batch_workspace(m, n, x.device)
    _check(load().compress_batch(m.h, mlp.h if mlp is not None else None, C.byref(grid.c),
                                 _ptr(x), n, _ptr(group_offsets), C.byref(params),
                                 C.byref(out.c), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def quantize_correct(grid: Grid, x, xhat, params: aeqc_params, mlp: Optional[MLP] = None,
                     latent=None, out: Optional[Compressed] = None,
                     outlier_capacity: Optional[int] = None, features: bool = False,
                     want_f: bool = False, ws=None, stream=None):
    """Stages 4-5 given decoded histograms xhat [n][ld] float32."""
    import torch
    n, P = x.shape
    L = latent.shape[1] if latent is not None else 0
    if out is None:
        cap = outlier_capacity if outlier_capacity is not None else max(1024, n * 4)
        out = Compressed(n, P, max(L, 1), torch.float32, x.device, cap, features and L > 0)
        if latent is not None:
            out.latent = latent
            out.c.latent = _ptr(latent)
    ldt = DTYPE_BF16 if (latent is not None and latent.dtype == torch.bfloat16) else DTYPE_F32
    f = torch.empty((n, P), dtype=torch.float64, device=x.device) if want_f else None
    if ws is None:
        ws = _workspace(load().quantize_correct_workspace_size(n), x.device)
    _check(load().quantize_correct(C.byref(grid.c), _ptr(x), _ptr(xhat), xhat.stride(0), n,
                                   C.byref(params), mlp.h if mlp is not None else None, ldt,
                                   L, C.byref(out.c), _ptr(f), _ptr(ws), ws.numel(),
                                   _stream(stream)))
    out.f = f
    return out


QC_NOALLOC_MAX_N = 262144  # AEQC_QC_NOALLOC_MAX_N


def quantize_correct_noalloc(grid: Grid, x, xhat, params: aeqc_params,
                             mlp: Optional[MLP] = None, latent=None,
                             out: Optional[Compressed] = None,
                             outlier_capacity: Optional[int] = None, features: bool = False,
                             want_f: bool = False, stream=None):
    """quantize_correct with the library's static scratch instead of a
    workspace (n <= QC_NOALLOC_MAX_N; calls must not overlap on the device).
    The output buffers are still the caller's: pass `out` (and no want_f) to
    make the call itself allocate nothing."""
    import torch
    n, P = x.shape
    L = latent.shape[1] if latent is not None else 0
    if out is None:
        cap = outlier_capacity if outlier_capacity is not None else max(1024, n * 4)
        out = Compressed(n, P, max(L, 1), torch.float32, x.device, cap, features and L > 0)
        if latent is not None:
            out.latent = latent
            out.c.latent = _ptr(latent)
    ldt = DTYPE_BF16 if (latent is not None and latent.dtype == torch.bfloat16) else DTYPE_F32
    f = torch.empty((n, P), dtype=torch.float64, device=x.device) if want_f else None
    _check(load().quantize_correct_noalloc(C.byref(grid.c), _ptr(x), _ptr(xhat),
                                           xhat.stride(0), n, C.byref(params),
                                           mlp.h if mlp is not None else None, ldt, L,
                                           C.byref(out.c), _ptr(f), _stream(stream)))
    out.f = f
    return out


def decompress_batch(m: Model, grid: Grid, comp: Compressed, params: aeqc_params,
                     group_offsets=None, f=None, ws=None, stream=None):
    import torch
    n = comp.n
    if f is None:
        f = torch.empty((n, m.P), dtype=torch.float64, device=comp.codes.device)
    if ws is None:
        ws = decompress_batch_workspace(m, n, comp.codes.device)
    _check(load().decompress_batch(m.h, C.byref(grid.c), C.byref(comp.c), n,
                                   _ptr(group_offsets), C.byref(params), _ptr(f), _ptr(ws),
                                   ws.numel(), _stream(stream)))
    return f


def _dtype_code(latent_dtype) -> int:
    import torch
    return DTYPE_BF16 if latent_dtype == torch.bfloat16 else DTYPE_F32


def batch_pack(comp: Compressed, stream=None) -> bytes:
    """Container blob of a compressed batch (codes, latents, multipliers,
    status, outlier list); synchronous."""
    lib = load()
    n, L = comp.latent.shape
    P = comp.codes.shape[1]
    dt = _dtype_code(comp.latent.dtype)
    cap = comp.c.outliers.capacity
    buf = C.create_string_buffer(lib.aeqc_batch_pack_size(n, P, L, dt, cap))
    written = C.c_size_t()
    _check(lib.aeqc_batch_pack(C.byref(comp.c), n, P, L, dt, buf, len(buf), C.byref(written),
                               _stream(stream)))
    return buf.raw[:written.value]


def batch_peek(blob: bytes) -> dict:
    """Validated header of a container blob (AeqcError ECORRUPT if invalid)."""
    n, outl = C.c_int64(), C.c_int64()
    P, L, dt = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().aeqc_batch_peek(blob, len(blob), C.byref(n), C.byref(P), C.byref(L),
                                  C.byref(dt), C.byref(outl)))
    return dict(n=n.value, P=P.value, L=L.value, latent_dtype=dt.value, outliers=outl.value)


def batch_unpack(blob: bytes, device, stream=None) -> Compressed:
    """Device buffers filled from a container blob; synchronous."""
    import torch
    h = batch_peek(blob)
    ldt = torch.bfloat16 if h["latent_dtype"] == DTYPE_BF16 else torch.float32
    comp = Compressed(h["n"], h["P"], h["L"], ldt, device, h["outliers"])
    _check(load().aeqc_batch_unpack(blob, len(blob), C.byref(comp.c), _stream(stream)))
    return comp


# --- product quantisation of the latents ----------------------------------------

def pq_train(z, k: int = 16, iters: int = 10, group_offsets=None, G: int = 1, table=None,
             ws=None, stream=None):
    """PQ table [G][L][k] float32 (device) from latents z [n][L] (float32 or
    bfloat16); rows of group g are group_offsets[g]:group_offsets[g+1]."""
    import torch
    n, L = z.shape
    lib = load()
    if table is None:
        table = torch.empty((G, L, k), dtype=torch.float32, device=z.device)
    need = lib.pq_train_workspace_size(G, L, k)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, z.device)
    _check(lib.pq_train(_ptr(z), _dtype_code(z.dtype), n, L, _ptr(group_offsets), G, k, iters,
                        _ptr(table), _ptr(ws), ws.numel(), _stream(stream)))
    return table


def pq_encode(z, table, group_offsets=None, codes=None, zq=None, want_codes: bool = True,
              stream=None):
    """(codes [n][L] uint8, zq [n][L] decoded latents or None)."""
    import torch
    n, L = z.shape
    G, _, k = table.shape
    if codes is None and want_codes:
        codes = torch.empty((n, L), dtype=torch.uint8, device=z.device)
    _check(load().pq_encode(_ptr(z), _dtype_code(z.dtype), n, L, _ptr(group_offsets), G, k,
                            _ptr(table), _ptr(codes), _ptr(zq), _stream(stream)))
    return codes, zq


def pq_decode(codes, table, latent_dtype, group_offsets=None, out=None, stream=None):
    """Latents [n][L] of latent_dtype from PQ codes and the table."""
    import torch
    n, L = codes.shape
    G, _, k = table.shape
    if out is None:
        out = torch.empty((n, L), dtype=latent_dtype, device=codes.device)
    _check(load().pq_decode(_ptr(codes), n, L, _ptr(group_offsets), G, k, _ptr(table),
                            _dtype_code(latent_dtype), _ptr(out), _stream(stream)))
    return out


# --- entropy coding of the residual codes ----------------------------------------

@dataclass
class RiceStreams:
    kparam: object   # [n] uint8
    nbits: object    # [n] uint32 (int32 storage)
    offsets: object  # [n + 1] int64, in words
    words: object    # [offsets[n]] int32 storage of uint32 words


def rice_encode(codes, ws=None, stream=None) -> RiceStreams:
    """Golomb-Rice streams of the residual codes [n][P] (device int16)."""
    import torch
    n, P = codes.shape
    dev = codes.device
    lib = load()
    kp = torch.empty(n, dtype=torch.uint8, device=dev)
    nb = torch.empty(n, dtype=torch.int32, device=dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    need = lib.rice_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, dev)
    _check(lib.rice_measure(_ptr(codes), n, P, _ptr(kp), _ptr(nb), _ptr(off), _ptr(ws),
                            ws.numel(), _stream(stream)))
    total = int(off[n].item())
    words = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    _check(lib.rice_pack(_ptr(codes), n, P, _ptr(kp), _ptr(off), _ptr(words), total,
                         _stream(stream)))
    return RiceStreams(kp, nb, off, words[:total])


def rice_decode(rs: RiceStreams, P: int, out=None, stream=None):
    """Residual codes [n][P] int16 from Golomb-Rice streams."""
    import torch
    n = rs.kparam.shape[0]
    if out is None:
        out = torch.empty((n, P), dtype=torch.int16, device=rs.kparam.device)
    _check(load().rice_unpack(_ptr(rs.words) if rs.words.numel() else None, rs.words.numel(),
                              _ptr(rs.offsets), _ptr(rs.kparam), n, P, _ptr(out),
                              _stream(stream)))
    return out


# --- NRMSE (Eq. (7)) and the error-bound search ------------------------------------

def nrmse_batch(x, f, per_hist: bool = False, stream=None):
    """(batch NRMSE as a float, per-histogram NRMSE tensor or None)."""
    import torch
    n, P = x.shape
    ph = torch.empty(n, dtype=torch.float64, device=x.device) if per_hist else None
    bt = torch.empty(1, dtype=torch.float64, device=x.device)
    ws = _workspace(load().nrmse_workspace_size(n), x.device)
    _check(load().nrmse_batch(_ptr(x), _ptr(f), n, P, _ptr(ph), _ptr(bt), _ptr(ws), ws.numel(),
                              _stream(stream)))
    return float(bt.item()), ph


def bound_search(m: Model, grid: Grid, x, params: aeqc_params, target: float,
                 tau_lo: float = 1e-6, tau_hi: float = 1e-1, probes: int = 12,
                 group_offsets=None, outlier_capacity: Optional[int] = None, stream=None):
    """(tau, nrmse): the largest probed pointwise bound whose batch NRMSE
    after compression and decompression stays within the target."""
    n = x.shape[0]
    cap = outlier_capacity if outlier_capacity is not None else max(1024, 16 * n)
    lib = load()
    ws = _workspace(lib.aeqc_bound_search_workspace_size(m.h, n, cap), x.device)
    t, e = C.c_double(), C.c_double()
    _check(lib.aeqc_bound_search(m.h, C.byref(grid.c), _ptr(x), n, _ptr(group_offsets),
                                 C.byref(params), target, tau_lo, tau_hi, probes, cap,
                                 C.byref(t), C.byref(e), _ptr(ws), ws.numel(), _stream(stream)))
    return t.value, e.value


# --- multi-GPU partitioning (host) ------------------------------------------

def partition_lpt(counts, n_ranks: int):
    """(owner [G] int32, load [n_ranks] int64): whole subdomains to ranks by
    the longest-processing-time rule on their histogram counts."""
    c = np.ascontiguousarray(counts, np.int64)
    owner = np.zeros(len(c), np.int32)
    load_ = np.zeros(int(n_ranks), np.int64)
    _check(load().aeqc_partition_lpt(c.ctypes.data if len(c) else None, len(c), int(n_ranks),
                                     owner.ctypes.data if len(c) else None, load_.ctypes.data))
    return owner, load_


def exclusive_scan(sizes):
    """offsets [n + 1]: where each rank's output starts, and the total."""
    sz = np.ascontiguousarray(sizes, np.int64)
    off = np.zeros(len(sz) + 1, np.int64)
    _check(load().aeqc_exclusive_scan(sz.ctypes.data if len(sz) else None, len(sz),
                                      off.ctypes.data))
    return off
