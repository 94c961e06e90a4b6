"""DIS tables in the reduced modes on the tensor cores (BF16, BF16 hi+lo, TF32).

The DIS observable is a plain product, O[r][d] = sum_{(k,i)} FK[d][(k,i)]
F[r][a_k][x_i] (the DIS rows of the paper's Table 1), and its adjoint the
product of gO with the transposed table, scattered onto the grid.  Pins:
small integers are exact in every mode (packing, gather map, tiles, scatter);
split-BF16 values with a lo part on one side are exact (both cross terms);
against the FP64 oracle every mode stays within its bound of S = sum |terms|;
a replica's result does not depend on R (K is never split).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu

TC = ("bf16", "bf16x3", "tf32")
# max |err| / S per mode for one product: the operand roundings (BF16 2 x 2^-8,
# TF32 2 x 2^-11, split BF16 3 x 2^-16, tests/test_gpu_tc.py) ...
BOUND = {"bf16": 2 ** -7, "tf32": 2 ** -9, "bf16x3": 3 * 2 ** -16}


def bound(prec, K):
    """... plus the FP32 accumulation of K products, at most K 2^-24 of S."""
    return BOUND[prec] + K * 2.0 ** -24


def dis_int(seed, nd, nfl, nx, nxg, R, lo=-3, hi=4):
    rng = np.random.default_rng(seed)
    flav = np.sort(rng.choice(14, nfl, replace=False)).astype(np.int32)
    fkv = np.zeros((nd, 14, nx))
    fkv[:, flav, :] = rng.integers(lo, hi, (nd, nfl, nx))
    xmap = np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32)
    t = W.DisTable(fkv, flav, xmap, nxg)
    F = rng.integers(lo, hi, (R, 14, nxg)).astype(np.float64)
    return t, F


def fwd(tab, F, prec, out=None):
    O = fk.conv(tab, torch.tensor(F, dtype=torch.float32, device="cuda"), prec, out=out)
    torch.cuda.synchronize()
    assert fk._lib.load().fk_device_status(1) == 0
    return O.double().cpu().numpy()


def bwd(tab, gO, prec, nxg, gF=None, accumulate=False):
    R = gO.shape[0]
    Fd = torch.zeros((R, 14, nxg), dtype=torch.float32, device="cuda")
    g = fk.conv_backward(tab, Fd, torch.tensor(gO, dtype=torch.float32, device="cuda"), prec, gF=gF,
                         accumulate=accumulate)
    torch.cuda.synchronize()
    assert fk._lib.load().fk_device_status(1) == 0
    return g.double().cpu().numpy()


SHAPES = [(1, 1, 1, 1, 1), (64, 9, 40, 40, 1), (300, 14, 64, 64, 130), (7, 5, 17, 50, 257),
          (257, 3, 3, 10, 3), (600, 12, 50, 50, 100)]


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("shape", SHAPES)
def test_dis_tc_exact_small_integers(prec, shape):
    """(ndata, active flavours, nx, grid, R): two data tiles (300, 257, 600 >
    256), ragged K, paired and odd replica tiles."""
    nd, nfl, nx, nxg, R = shape
    t, F = dis_int(sum(shape), nd, nfl, nx, nxg, R)
    tab = fk.Table.from_workload(t, precs=(prec,))
    O_ref, _ = oracle.dis(t, F)
    assert np.array_equal(fwd(tab, F, prec), O_ref)
    gO = np.random.default_rng(7).integers(-3, 4, (R, nd)).astype(np.float64)
    assert np.array_equal(bwd(tab, gO, prec, nxg), oracle.dis_grad(t, gO))


@pytest.mark.parametrize("side", ["F", "FK"])
def test_dis_bf16x3_cross_terms_exact(side):
    """hi + lo held exactly on one side (h = +-1, +-2, l = k 2^-10, |k| <= 3),
    integers in -1..1 on the other: BF16X3 is exact, plain BF16 is not."""
    nd, nfl, nx, nxg, R = 37, 9, 40, 50, 130
    rng = np.random.default_rng(5 + len(side))

    def split(shape):
        h = rng.integers(1, 3, shape) * rng.choice([-1.0, 1.0], shape)
        return h + rng.integers(-3, 4, shape) * 2.0 ** -10

    flav = np.sort(rng.choice(14, nfl, replace=False)).astype(np.int32)
    fkv = np.zeros((nd, 14, nx))
    fkv[:, flav, :] = split((nd, nfl, nx)) if side == "FK" else rng.integers(-1, 2, (nd, nfl, nx))
    t = W.DisTable(fkv, flav, np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32), nxg)
    F = split((R, 14, nxg)) if side == "F" else rng.integers(-1, 2, (R, 14, nxg)).astype(np.float64)
    tab = fk.Table.from_workload(t, precs=("bf16x3", "bf16"))
    O_ref, _ = oracle.dis(t, F)
    assert np.array_equal(fwd(tab, F, "bf16x3"), O_ref)
    assert not np.array_equal(fwd(tab, F, "bf16"), O_ref)
    if side == "FK":  # the adjoint's MMA operands are gO and the table
        gO = rng.integers(-2, 3, (R, nd)).astype(np.float64)
        g_ref = oracle.dis_grad(t, gO)
        assert np.array_equal(bwd(tab, gO, "bf16x3", nxg), g_ref)
        assert not np.array_equal(bwd(tab, gO, "bf16", nxg), g_ref)


@pytest.mark.parametrize("prec", TC)
def test_dis_tc_accuracy(prec):
    """Config-0 shaped table at R = 100 and the DIS tables of the global set:
    error against the FP64 oracle within the mode's bound of S."""
    t0, _ = W.config0()
    x = W.xgrid(40, 1e-7)
    rng = np.random.default_rng(3)
    F0 = W.pdf_replicas(x, W.pdf_params(rng), 100, rng)
    g = W.config3(R=20, scale=0.3)
    cases = [(t0, F0)] + [(t, g.F) for t in g.tables if not hasattr(t, "ca")][:4]
    worst = 0.0
    for t, F in cases:
        tab = fk.Table.from_workload(t, precs=(prec,))
        O_ref, S = oracle.dis(t, F)
        err = float((np.abs(fwd(tab, F, prec) - O_ref) / S).max())
        assert err <= bound(prec, len(t.flav) * t.nx), (prec, err)
        gO = rng.standard_normal((F.shape[0], t.ndata))
        g_ref = oracle.dis_grad(t, gO)
        scale = oracle.dis_grad(W.DisTable(np.abs(t.fk), t.flav, t.xmap, t.nxg), np.abs(gO))
        gerr = float((np.abs(bwd(tab, gO, prec, t.nxg) - g_ref) / np.maximum(scale, 1e-300)).max())
        assert gerr <= bound(prec, t.ndata), (prec, gerr)
        worst = max(worst, err, gerr)
    print(prec, "DIS max err/S", worst)


@pytest.mark.parametrize("prec", TC)
def test_dis_tc_replica_independent_of_R(prec):
    t, F = dis_int(11, 200, 9, 40, 50, 300, lo=-50, hi=50)
    F = F * 0.0137  # non-integer values: results round, the order must not change
    tab = fk.Table.from_workload(t, precs=(prec,))
    full = fwd(tab, F, prec)
    assert np.array_equal(full[37:37 + 64], fwd(tab, F[37:37 + 64], prec))
    assert np.array_equal(full[299:300], fwd(tab, F[299:300], prec))


def test_dis_tc_ldo_and_accumulate():
    g = W.config3(R=9, scale=0.1)
    dis = [t for t in g.tables if not hasattr(t, "ca")][:3]
    ntot = sum(t.ndata for t in dis)
    out = torch.full((9, ntot + 2), float("nan"), device="cuda")
    gF = torch.zeros(g.F.shape, dtype=torch.float32, device="cuda")
    Fd = torch.tensor(g.F, dtype=torch.float32, device="cuda")
    off = 0
    g_ref = np.zeros_like(g.F)
    rng = np.random.default_rng(2)
    for t in dis:
        tab = fk.Table.from_workload(t, precs=("bf16x3",))
        fk.conv(tab, Fd, "bf16x3", out=out[:, off:off + t.ndata])
        gO = rng.standard_normal((9, t.ndata))
        fk.conv_backward(tab, Fd, torch.tensor(gO, dtype=torch.float32, device="cuda"), "bf16x3", gF=gF,
                         accumulate=True)
        g_ref += oracle.dis_grad(t, gO)
        O_ref, S = oracle.dis(t, g.F)
        torch.cuda.synchronize()
        assert (np.abs(out[:, off:off + t.ndata].double().cpu().numpy() - O_ref) / S).max() <= BOUND["bf16x3"]
        off += t.ndata
    assert torch.isnan(out[:, ntot:]).all()
    got = gF.double().cpu().numpy()
    assert np.abs(got - g_ref).max() <= 2 ** -14 * np.abs(g_ref).max()
