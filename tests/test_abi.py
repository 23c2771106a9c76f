"""The C-ABI library loads and exports every function include/aeqc.h declares
(no compute calls: runs without a GPU), and host-side argument checks fail
loudly before anything is launched."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aeqc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\**\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_10733_gb300 import aeqc, build
    build.build()
    return aeqc.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ae_encode", "ae_decode", "residual_quantize", "residual_dequantize",
              "qoi_moments", "qoi_correct", "compress_batch", "decompress_batch",
              "ae_train_step", "quantize_correct", "mlp_train_step", "mlp_predict"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2212_10733_gb300 import aeqc
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared names
    assert set(aeqc.SYMBOLS) == set(declared_functions())


def test_params_default_and_version(lib):
    from paper_2212_10733_gb300 import aeqc
    p = aeqc.params_default()
    assert p.tau == 1e-4 and p.alpha == 0.5 and p.step_s == 1.0 and p.tol == 1e-12
    assert p.max_iter == 50 and p.r2_max_iter == 400 and p.warm_iters == 2
    assert lib.aeqc_version().decode().startswith("aeqc")


def test_argument_errors_are_caught_on_the_host(lib):
    from paper_2212_10733_gb300 import aeqc, synth
    p = aeqc.params_default(tau=-1.0)
    rc = lib.residual_quantize(None, None, 1536, 4, 1521, C.byref(p), None, None, None, None,
                               None, None)
    assert rc == aeqc.EINVAL
    assert b"tau" in lib.aeqc_last_error()
    p = aeqc.params_default()
    rc = lib.residual_quantize(None, None, 10, 4, 1521, C.byref(p), None, None, None, None,
                               None, None)
    assert rc == aeqc.EINVAL  # ld < P
    vpar, vperp, vol = synth.grid_arrays(n_par=65)
    g = aeqc.Grid(vpar, vperp, vol)
    rc = lib.qoi_moments(C.byref(g.c), None, 1, None, None)
    assert rc == aeqc.EINVAL and b"n_par" in lib.aeqc_last_error()
    # empty batches are valid no-ops
    vpar, vperp, vol = synth.grid_arrays()
    g = aeqc.Grid(vpar, vperp, vol)
    assert lib.qoi_moments(C.byref(g.c), None, 0, None, None) == aeqc.OK
    # model descriptors are validated before any allocation
    d = aeqc.aeqc_model_desc(1521, 100, 16, 1, 0, 0, 1, 0)
    h = C.c_void_p()
    assert lib.aeqc_model_create(C.byref(d), C.byref(h)) == aeqc.EINVAL
    assert b"H=100" in lib.aeqc_last_error()


def test_noalloc_rejects_batches_above_its_static_limit(lib):
    from paper_2212_10733_gb300 import aeqc, synth
    vpar, vperp, vol = synth.grid_arrays()
    g = aeqc.Grid(vpar, vperp, vol)
    p = aeqc.params_default(kernel=aeqc.KERNEL_FAST)
    n = aeqc.QC_NOALLOC_MAX_N + 1
    rc = lib.quantize_correct_noalloc(C.byref(g.c), None, None, 1536, n, C.byref(p), None, 0,
                                      0, None, None, None)
    assert rc == aeqc.EINVAL and b"static scratch limit" in lib.aeqc_last_error()
    header = open(HEADER).read()
    assert re.search(r"#define AEQC_QC_NOALLOC_MAX_N %d\b" % aeqc.QC_NOALLOC_MAX_N, header)
