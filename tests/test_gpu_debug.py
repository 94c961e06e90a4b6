"""The debug build (libfk_debug.so, FK_DEBUG=1) on small odd shapes.

Index checks in the kernels record the first failed check and skip the
access; per-call scratch buffers carry guard bytes verified when they are
released.  A child process loads the debug build, runs every path (hadronic
and DIS forward and adjoint in all modes, the hadronic forward's dense form,
the dense product, chi^2) on the
shapes nx = 1, 17, 33, ndata = 1, 129, one channel, R = 1, 3, 257, compares
with the FP64 oracle and then requires fk_debug_status to report no failed
check; fk_debug_selftest shows that a failed check is reported.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

CHILD = r'''
import numpy as np, torch, ctypes
import oracle, paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import _lib, workloads as W
assert _lib.path().endswith("libfk_debug.so")
lib = _lib.load()
tol = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 2 ** -7, "bf16x3": 3 * 2 ** -16, "tf32": 2 ** -9, "fp64tc": 1e-12}
worst = 0.0
for (nd, nc, nx, R) in [(1, 1, 1, 1), (129, 1, 17, 3), (1, 5, 33, 257), (129, 3, 33, 1), (7, 1, 17, 257)]:
    rng = np.random.default_rng(nd + nc + nx + R)
    x = W.xgrid(nx, 1e-6)
    F = W.pdf_replicas(x, W.pdf_params(rng), R, rng)
    gO = rng.standard_normal((R, nd))
    for t in (W.had_table(rng, nd, nc, x), W.dis_table(rng, nd, min(nc, 14), x)):
        O_ref, S = oracle.conv(t, F)
        g_ref = oracle.conv_grad(t, F, gO)
        for prec in ("fp64", "fp32", "bf16", "bf16x3", "tf32", "fp64tc"):
            tab = fk.Table.from_workload(t, precs=(prec,))
            dt = torch.float64 if prec in ("fp64", "fp64tc") else torch.float32
            Fd = torch.tensor(F, dtype=dt, device="cuda")
            O = fk.conv(tab, Fd, prec).double().cpu().numpy()
            err = float((np.abs(O - O_ref) / S).max())
            assert err <= tol[prec], (nd, nc, nx, R, prec, err)
            g = fk.conv_backward(tab, Fd, torch.tensor(gO, dtype=dt, device="cuda"), prec).double().cpu().numpy()
            assert np.all(np.isfinite(g))
            worst = max(worst, err)
            if prec in ("bf16", "bf16x3", "tf32") and hasattr(t, "ca"):
                # saved forward products: the same O and gF bit for bit
                sv = fk.saved_buffer(tab, R, prec)
                O2 = fk.conv(tab, Fd, prec, save=sv).double().cpu().numpy()
                g2 = fk.conv_backward(tab, Fd, torch.tensor(gO, dtype=dt, device="cuda"), prec,
                                      saved=sv).double().cpu().numpy()
                assert np.array_equal(O2, O) and np.array_equal(g2, g), (nd, nc, nx, R, prec)
# the dense form of the hadronic forward (PDF matrix built in shared memory)
for (nd, nc, nx, R) in [(1, 1, 1, 1), (129, 3, 17, 3), (300, 5, 33, 257)]:
    rng = np.random.default_rng(nd + nc + nx + R + 1)
    x = W.xgrid(nx, 1e-6)
    F = W.pdf_replicas(x, W.pdf_params(rng), R, rng)
    t = W.had_table(rng, nd, nc, x)
    O_ref, S = oracle.conv(t, F)
    for prec in ("bf16", "bf16x3", "tf32"):
        tab = fk.Table.from_workload(t, precs=(prec,), form="lumi")
        O = fk.conv(tab, torch.tensor(F, dtype=torch.float32, device="cuda"), prec).double().cpu().numpy()
        assert (np.abs(O - O_ref) / S).max() <= tol[prec] + 1600 * 2.0 ** -24, (nd, nc, nx, R, prec)
L = np.random.default_rng(1).standard_normal((3, 300))
fkd = np.random.default_rng(2).standard_normal((129, 300))
O_ref, S = oracle.dense(fkd, L)
for prec in ("fp32", "bf16x3", "fp64tc"):
    tab = fk.Table.dense(fkd, precs=(prec,))
    dt = torch.float64 if prec == "fp64tc" else torch.float32
    O = fk.dense_conv(tab, torch.tensor(L, dtype=dt, device="cuda"), prec).double().cpu().numpy()
    assert (np.abs(O - O_ref) / S).max() <= tol[prec]
blocks = [np.eye(1) * 2.0, np.diag(np.linspace(1, 2, 33)) + 0.1]
cov = fk.Cov(blocks)
Od = torch.tensor(np.random.default_rng(3).standard_normal((257, 34)), device="cuda")
c, gc = fk.chi2(cov, Od, torch.zeros(34, dtype=torch.float64, device="cuda"))
torch.cuda.synchronize()
code, idx = ctypes.c_int(-1), ctypes.c_longlong(-1)
assert lib.fk_debug_status(0, ctypes.byref(code), ctypes.byref(idx)) == 0
assert code.value == 0, ("failed check", code.value, idx.value)
assert lib.fk_debug_selftest() == 0
print("debug build clean, worst err/S", worst)
'''


def test_debug_build_clean_on_small_odd_shapes():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FK_DEBUG="1")
    out = subprocess.run([sys.executable, "-c", CHILD], cwd=root, env=env, capture_output=True, text=True,
                         timeout=1200)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "debug build clean" in out.stdout
