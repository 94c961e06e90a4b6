"""fk_had_conv_noalloc: the hadronic convolution for callers that may not
allocate device memory while they run (their GPU memory belongs to another
allocator or is capped, or they cannot afford an allocation in a tight loop).
Its partial sums live in a static device array instead of per-call scratch.

Checked through the C ABI on three calls in a row (a streaming call with
R = 1, then the many-replica kernel's 16-wide replica tile with R = 3, then
its wide tile with R = 37 on another table, so each call reuses the array the
previous one left behind): bit-equal to fk_had_conv on the same inputs (the
launches and their summation order are the same), and within the tolerances
of the other parity tests of the FP64 oracle: 1e-12 (FP64) and 1e-5 (FP32) of
the sum of |terms|.  This file is collected last so a failure here never
hides others.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import _lib
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _call(name, tab, F, O, prec):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(_lib.load(), name)(tab.handle, ctypes.c_void_p(F.data_ptr()), F.shape[0],
                                    ctypes.c_void_p(O.data_ptr()), 0, _lib.PRECS[prec], stream)
    assert rc == 0, (name, _lib.load().fk_last_error_message())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_fk_had_conv_on_two_calls(prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    cases = [W.config1(R=1), W.config1(R=3, seed=98, ndata=90, nc=30, nx=20),
             W.config1(R=37, seed=99, ndata=150, nc=40, nx=25)]
    for t, F in cases:
        tab = fk.Table.from_workload(t, precs=(prec,))
        Fd = torch.tensor(F, dtype=dt, device="cuda")
        O_ref = torch.empty((F.shape[0], t.ndata), dtype=dt, device="cuda")
        O_new = torch.full_like(O_ref, float("nan"))
        _call("fk_had_conv", tab, Fd, O_ref, prec)
        _call("fk_had_conv_noalloc", tab, Fd, O_new, prec)
        torch.cuda.synchronize()
        assert torch.equal(O_new, O_ref)
        want, S = oracle.had(t, F)
        err = np.abs(O_new.double().cpu().numpy() - want)
        assert np.all(err <= TOL[prec] * S), (err / S).max()


def test_noalloc_rejects_oversized_call():
    t, F = W.config1(R=1)
    tab = fk.Table.from_workload(t, precs=("fp64",))
    R = 2000  # 60 channel splits x 2000 replicas x 200 points x 8 B >> 8 MiB
    Fd = torch.zeros((R, 14, t.nxg), dtype=torch.float64, device="cuda")
    O = torch.zeros((R, t.ndata), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = _lib.load()
    rc = lib.fk_had_conv_noalloc(tab.handle, ctypes.c_void_p(Fd.data_ptr()), R,
                                 ctypes.c_void_p(O.data_ptr()), 0, _lib.FK_FP64, stream)
    assert rc == _lib.FK_EINVAL
    assert b"bytes of partial sums" in lib.fk_last_error_message()
