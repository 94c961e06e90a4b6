"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (spec contract): FP64 mode 1e-12, FP32 mode 1e-5, relative to
S[r][d] = sum of |terms| of the observable (the scale of any summation error;
plain relative error is meaningless for signed hadronic tables whose terms
cancel).  All-positive DIS tables also meet the plain relative bound.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
DT = {"fp64": torch.float64, "fp32": torch.float32}


def dev(a, prec="fp64"):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=DT[prec])


def run_conv(tab, F, prec):
    out = fk.conv(tab, dev(F, prec), prec)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def assert_scaled(got, want, S, tol, what=""):
    err = np.abs(got - want)
    bound = tol * np.maximum(S, np.finfo(np.float64).tiny)
    bad = err > bound
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} outside {tol}*S; "
                           f"max err/S = {(err / np.maximum(S, 1e-300)).max():.3e}")


class Tiny:
    def __init__(self, fk_, ca=None, cb=None, xmap=None, nxg=None, flav=None):
        self.fk = np.asarray(fk_, np.float64)
        nx = self.fk.shape[-1]
        self.xmap = np.arange(nx, dtype=np.int32) if xmap is None else np.asarray(xmap, np.int32)
        self.nxg = nx if nxg is None else nxg
        if ca is not None:
            self.ca, self.cb = np.asarray(ca, np.int32), np.asarray(cb, np.int32)
        if flav is not None:
            self.flav = np.asarray(flav, np.int32)

    def compact(self):
        return np.ascontiguousarray(self.fk[:, self.flav, :])


# ------------------------------------------------------------ config 0 ----

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config0_dis(prec):
    t, F = W.config0()
    O_ref, S = oracle.dis(t, F)
    tab = fk.Table.from_workload(t)
    O = run_conv(tab, F, prec)
    assert_scaled(O, O_ref, S, TOL[prec], "cfg0")
    assert np.all(np.abs(O - O_ref) <= TOL[prec] * np.abs(O_ref))  # all-positive terms


# ------------------------------------------------------------ config 1 ----

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("R", [1, 100])
def test_config1_had(prec, R):
    t, F = W.config1(R=R)
    O_ref, S = oracle.had(t, F)
    tab = fk.Table.from_workload(t)
    O = run_conv(tab, F, prec)
    assert_scaled(O, O_ref, S, TOL[prec], f"cfg1 R={R}")


# ------------------------------------------------------ exact integers ----

def _int_had(seed, nd, nc, nx, nxg, R):
    rng = np.random.default_rng(seed)
    ca, cb = W.channels(rng, nc)
    fk_ = rng.integers(-3, 4, (nd, nc, nx, nx)).astype(np.float64)
    xmap = np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32)
    F = rng.integers(-3, 4, (R, 14, nxg)).astype(np.float64)
    return Tiny(fk_, ca, cb, xmap, nxg), F


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("R", [1, 3, 7])
def test_had_exact_small_integers(prec, R):
    """All partial sums are integers below 2^24: every path must be exact."""
    t, F = _int_had(31 + R, nd=5, nc=6, nx=5, nxg=9, R=R)
    O_ref, _ = oracle.had(t, F)
    tab = fk.Table.had(t.fk, t.ca, t.cb, t.xmap, t.nxg)
    assert np.array_equal(run_conv(tab, F, prec), O_ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("R", [1, 9])
def test_dis_exact_small_integers(prec, R):
    rng = np.random.default_rng(40 + R)
    nd, nx, nxg = 11, 7, 12
    flav = np.array([0, 3, 4, 9, 13], np.int32)
    fk_ = np.zeros((nd, 14, nx))
    fk_[:, flav] = rng.integers(-4, 5, (nd, len(flav), nx))
    xmap = np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32)
    F = rng.integers(-4, 5, (R, 14, nxg)).astype(np.float64)
    t = Tiny(fk_, xmap=xmap, nxg=nxg, flav=flav)
    O_ref, _ = oracle.dis(t, F)
    tab = fk.Table.dis(t.compact(), flav, xmap, nxg)
    assert np.array_equal(run_conv(tab, F, prec), O_ref)


# ------------------------------------------------------- ragged shapes ----

RAGGED = [  # (ndata, nc, nx, R)
    (1, 1, 1, 1), (1, 1, 17, 3), (129, 3, 17, 1), (129, 5, 33, 5), (7, 196, 3, 257),
    (65, 13, 64, 66), (200, 60, 30, 4), (3, 2, 2, 130),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", RAGGED)
def test_had_ragged(prec, shape):
    nd, nc, nx, R = shape
    rng = np.random.default_rng(nd * 1000 + nc * 10 + nx + R)
    x = W.xgrid(nx, 1e-6)
    t = W.had_table(rng, nd, nc, x)
    F = W.pdf_replicas(x, W.pdf_params(rng), R, rng)
    O_ref, S = oracle.had(t, F)
    tab = fk.Table.from_workload(t)
    assert_scaled(run_conv(tab, F, prec), O_ref, S, TOL[prec], str(shape))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (129, 14, 33, 5), (600, 9, 50, 100), (3, 5, 64, 1)])
def test_dis_ragged(prec, shape):
    nd, nact, nx, R = shape
    rng = np.random.default_rng(nd + nact + nx + R)
    x = W.xgrid(nx, 1e-7)
    t = W.dis_table(rng, nd, nact, x)
    F = W.pdf_replicas(x, W.pdf_params(rng), R, rng)
    O_ref, S = oracle.dis(t, F)
    tab = fk.Table.from_workload(t)
    assert_scaled(run_conv(tab, F, prec), O_ref, S, TOL[prec], str(shape))


def test_shared_grid_xmap():
    """Tables on subsets of a 50-point master grid (the global-fit layout)."""
    g = W.config3(R=4, scale=0.05)
    for t in g.tables[:8]:
        O_ref, S = oracle.conv(t, g.F)
        tab = fk.Table.from_workload(t)
        for prec in ("fp64", "fp32"):
            assert_scaled(run_conv(tab, g.F, prec), O_ref, S, TOL[prec], "xmap")


# ------------------------------------------------------------ adjoint ----

def _grad_scale(t, F, gO):
    """sum of |terms| of each gradient entry: the oracle's gradient of |FK|
    with |F| and |gO| (every term of the adjoint is a product of those)."""
    a = Tiny(np.abs(t.fk), getattr(t, "ca", None), getattr(t, "cb", None), t.xmap, t.nxg)
    return oracle.conv_grad(a, np.abs(F), np.abs(gO))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(200, 60, 30, 100), (17, 3, 33, 1), (129, 196, 5, 65), (5, 1, 64, 3)])
def test_had_backward(prec, shape):
    nd, nc, nx, R = shape
    rng = np.random.default_rng(sum(shape))
    x = W.xgrid(nx, 1e-6)
    t = W.had_table(rng, nd, nc, x)
    F = W.pdf_replicas(x, W.pdf_params(rng), R, rng)
    gO = rng.standard_normal((R, nd))
    ref = oracle.had_grad(t, F, gO)
    S = _grad_scale(t, F, gO)
    tab = fk.Table.from_workload(t)
    gF = fk.conv_backward(tab, dev(F, prec), dev(gO, prec), prec)
    torch.cuda.synchronize()
    assert_scaled(gF.double().cpu().numpy(), ref, S, TOL[prec], f"bwd {shape}")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_backward_accumulates_over_tables(prec):
    g = W.config3(R=5, scale=0.05)
    gF_ref = np.zeros_like(g.F)
    S = np.zeros_like(g.F)
    gF = torch.zeros(g.F.shape, dtype=DT[prec], device="cuda")
    Fd = dev(g.F, prec)
    rng = np.random.default_rng(2)
    for t in g.tables[:10]:
        gO = rng.standard_normal((5, t.ndata))
        gF_ref += oracle.conv_grad(t, g.F, gO)
        S += _grad_scale(t, g.F, gO)
        tab = fk.Table.from_workload(t)
        fk.conv_backward(tab, Fd, dev(gO, prec), prec, gF=gF, accumulate=True)
    torch.cuda.synchronize()
    assert_scaled(gF.double().cpu().numpy(), gF_ref, S, TOL[prec], "accumulate")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dis_backward(prec):
    g = W.config3(R=7, scale=0.2)
    t = [t for t in g.tables if not hasattr(t, "ca")][0]
    rng = np.random.default_rng(3)
    gO = rng.standard_normal((7, t.ndata))
    ref = oracle.dis_grad(t, gO)
    S = _grad_scale(t, g.F, gO)
    tab = fk.Table.from_workload(t)
    gF = fk.conv_backward(tab, dev(g.F, prec), dev(gO, prec), prec)
    torch.cuda.synchronize()
    assert_scaled(gF.double().cpu().numpy(), ref, S, TOL[prec], "dis bwd")


# ---------------------------------------------------------- determinism ----

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_replica_result_independent_of_batch(prec):
    """A replica's observables do not depend on which other replicas share
    the launch (needed for bit-exact continuous batching)."""
    t, F = W.config1(R=300)
    tab = fk.Table.from_workload(t)
    full = run_conv(tab, F, prec)
    part = run_conv(tab, F[37:37 + 64], prec)
    assert np.array_equal(full[37:37 + 64], part)
    small = run_conv(tab, F[5:8], prec)       # replica tile of 16 instead of 64 (32 in FP64)
    again = run_conv(tab, F[5:8], prec)
    assert np.array_equal(small, again)
    assert np.array_equal(full[5:8], small)


# ---------------------------------------------------------------- errors ----

def test_argument_errors_are_reported():
    t, F = W.config0()
    tab = fk.Table.from_workload(t, precs=("fp64",))
    with pytest.raises(fk.FKError, match="unsupported"):
        fk.conv(tab, dev(F, "fp32"), "fp32")
    with pytest.raises(fk.FKError, match="invalid"):
        fk._lib.call("fk_had_conv", tab.handle, fk._p(dev(F)), 1, fk._p(dev(F)), 0, 0, None)
    with pytest.raises(fk.FKError, match="invalid"):
        fk._lib.call("fk_dis_conv", tab.handle, fk._p(dev(F)), 0, fk._p(dev(F)), 0, 0, None)
    with pytest.raises(fk.FKError, match="invalid"):
        fk.Table.had(np.zeros((1, 2, 3, 3)), [0, 0], [1, 1])  # duplicate channel
    with pytest.raises(fk.FKError, match="invalid"):
        fk.Table.had(np.zeros((1, 1, 3, 3)), [0], [1], xmap=[0, 0, 1], nx_grid=4)
