"""Host-side checks of the C ABI: the library loads and exports every symbol
include/fk.h declares; argument errors are caught before any CUDA call."""
import ctypes
import os
import re

import pytest

import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fk_\w+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    need = {"fk_dis_conv", "fk_had_conv", "fk_conv_backward", "fk_chi2", "fk_serve_submit",
            "fk_serve_poll", "fk_table_create_had", "fk_table_create_dis", "fk_cov_create"}
    assert need <= declared()


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert not missing, missing
    bound = set(_lib.SIGNATURES) | set(_lib.STRING_FUNCS) | set(_lib.U64_FUNCS)
    assert declared() <= bound, declared() - bound


def test_version_and_strerror():
    lib = _lib.load()
    assert lib.fk_version() >= 100
    assert lib.fk_strerror(_lib.FK_EINVAL) == b"invalid argument"
    assert lib.fk_strerror(12345) == b"unknown status"


@pytest.mark.parametrize("bad", [
    dict(fk_shape=(0, 1, 3, 3)),                 # ndata < 1
    dict(fk_shape=(1, 1, 65, 65)),               # nx too large
    dict(ca=[14], cb=[0]),                       # flavour out of range
    dict(ca=[1, 1], cb=[2, 2], fk_shape=(1, 2, 3, 3)),  # duplicate channel
    dict(precs=()),                              # empty mask
])
def test_table_argument_errors_need_no_gpu(bad):
    import numpy as np
    shape = bad.get("fk_shape", (1, 1, 3, 3))
    with pytest.raises(fk.FKError) as e:
        fk.Table.had(np.zeros(shape), bad.get("ca", [0] * shape[1]), bad.get("cb", [1] * shape[1]),
                     precs=bad.get("precs", ("fp32",)))
    assert e.value.status == _lib.FK_EINVAL


def test_null_pointer_calls_are_rejected():
    lib = _lib.load()
    assert lib.fk_had_conv(None, None, 1, None, 0, 0, None) == _lib.FK_EINVAL
    assert lib.fk_conv_backward(None, None, None, 0, 1, None, 0, 0, None) == _lib.FK_EINVAL
    assert lib.fk_chi2(None, None, None, 1, None, None, 0, None) == _lib.FK_EINVAL
    assert lib.fk_table_destroy(None) == 0
    assert lib.fk_cov_size(None) == 0


@pytest.mark.parametrize("shape,precs", [((0, 5), ("fp32",)), ((2, 0), ("fp32",)), ((2, 5), ())])
def test_dense_table_argument_errors_need_no_gpu(shape, precs):
    import numpy as np
    with pytest.raises(fk.FKError) as e:
        fk.Table.dense(np.zeros(shape), precs=precs)
    assert e.value.status == _lib.FK_EINVAL


def test_dense_and_luminosity_reject_null_handles():
    lib = _lib.load()
    assert lib.fk_dense_conv(None, None, 1, None, 0, 0, None) == _lib.FK_EINVAL
    assert lib.fk_luminosity(None, None, 1, None, 0, None) == _lib.FK_EINVAL


def test_dense_table_k_limit_needs_no_gpu():
    import ctypes
    import numpy as np
    lib = _lib.load()
    buf = np.zeros(4)
    out = ctypes.c_void_p()
    # the limit is checked before the table is read
    assert lib.fk_table_create_dense(buf.ctypes.data_as(ctypes.c_void_p), 1, (1 << 30) + 1,
                                     1 << _lib.FK_FP32, ctypes.byref(out)) == _lib.FK_EINVAL


def test_debug_build_exports_and_release_reports_no_debug():
    """libfk_debug.so (FK_DEBUG defined) exports the same boundary; the
    release library answers the debug queries with FK_EUNSUPPORTED, without
    touching a GPU."""
    from paper_1909_10547_b300 import build as _b
    path = _b.build(debug=True)
    dbg = ctypes.CDLL(path)
    missing = [n for n in sorted(declared()) if not hasattr(dbg, n)]
    assert not missing, missing
    lib = _lib.load()
    code, idx = ctypes.c_int(-1), ctypes.c_longlong(-1)
    assert lib.fk_debug_status(0, ctypes.byref(code), ctypes.byref(idx)) == _lib.FK_EUNSUPPORTED
    assert code.value == 0 and idx.value == 0
    assert lib.fk_debug_selftest() == _lib.FK_EUNSUPPORTED


def test_form_flags_are_checked_on_the_host():
    """FK_TABLE_FACTORED and FK_TABLE_LUMI: at most one, hadronic tables only
    (rejected before any device work)."""
    import numpy as np
    lib = _lib.load()
    out = ctypes.c_void_p()
    fkv = np.zeros((1, 1, 3, 3))
    ca, cb = np.zeros(1, np.int32), np.ones(1, np.int32)
    both = (1 << _lib.FK_FP32) | _lib.FK_TABLE_FACTORED | _lib.FK_TABLE_LUMI
    assert lib.fk_table_create_had(fkv.ctypes.data, 1, ca.ctypes.data, cb.ctypes.data, 1, 3, None, 3, both,
                                   ctypes.byref(out)) == _lib.FK_EINVAL
    fd, flav = np.zeros((1, 1, 3)), np.zeros(1, np.int32)
    assert lib.fk_table_create_dis(fd.ctypes.data, 1, flav.ctypes.data, 1, 3, None, 3,
                                   (1 << _lib.FK_FP32) | _lib.FK_TABLE_LUMI, ctypes.byref(out)) == _lib.FK_EINVAL
    with pytest.raises(ValueError):
        fk.Table.from_workload(type("D", (), {"compact": lambda s: fd, "flav": flav, "xmap": None, "nxg": 3})(),
                               precs=("fp32",), form="lumi")


def test_probe_argument_errors_need_no_gpu():
    lib = _lib.load()
    assert lib.fk_mma_probe(8, 10, 0, ctypes.c_void_p(1), None) == _lib.FK_EINVAL     # n not a multiple of 16
    assert lib.fk_mma_probe(272, 10, 0, ctypes.c_void_p(1), None) == _lib.FK_EINVAL   # n > 256
    assert lib.fk_mma_probe(64, 0, 0, ctypes.c_void_p(1), None) == _lib.FK_EINVAL     # iters < 1
    assert lib.fk_mma_probe(64, 10, 2, ctypes.c_void_p(1), None) == _lib.FK_EINVAL    # fill not 0 or 1
    assert lib.fk_mma_probe(64, 10, 0, None, None) == _lib.FK_EINVAL                  # no output
    assert lib.fk_fma_probe(_lib.FK_BF16, 1, 1, ctypes.c_void_p(1), None) == _lib.FK_EINVAL


def test_saved_product_argument_errors_need_no_gpu():
    lib = _lib.load()
    n = ctypes.c_size_t(7)
    assert lib.fk_saved_size(None, 1, _lib.FK_BF16X3, ctypes.byref(n)) == _lib.FK_EINVAL  # no table
    assert n.value == 0
    assert lib.fk_saved_size(None, 1, _lib.FK_BF16X3, None) == _lib.FK_EINVAL            # no output
    p = ctypes.c_void_p(16)
    assert lib.fk_had_conv_save(None, p, 1, p, 0, p, 1 << 20, _lib.FK_BF16X3, None) == _lib.FK_EINVAL
    assert lib.fk_conv_backward_saved(None, p, p, 0, 1, p, 1 << 20, p, 0, _lib.FK_BF16X3,
                                      None) == _lib.FK_EINVAL


def test_chi2_white_argument_errors_need_no_gpu():
    lib = _lib.load()
    p = ctypes.c_void_p(16)
    assert lib.fk_chi2_white(None, 0, p, 4, 2, p, None, 0, _lib.FK_FP64, None) == _lib.FK_EINVAL  # no Z
    assert lib.fk_chi2_white(p, 0, p, 0, 2, p, None, 0, _lib.FK_FP64, None) == _lib.FK_EINVAL     # n < 1
    assert lib.fk_chi2_white(p, 3, p, 4, 2, p, None, 0, _lib.FK_FP64, None) == _lib.FK_EINVAL     # ldz < n
    assert lib.fk_chi2_white(p, 0, p, 4, 2, p, p, 2, _lib.FK_FP64, None) == _lib.FK_EINVAL        # ldg < n
    assert lib.fk_chi2_white(p, 0, p, 4, 2, p, None, 0, 99, None) == _lib.FK_EINVAL               # precision
