"""Tensor-core (tcgen05) modes vs the FP64 oracle.

Exactness pins: with small-integer tables and PDFs every product and partial
sum is an exact integer in BF16/TF32 operands with FP32 accumulation, so all
three modes must reproduce the oracle bit for bit; that pins the packing,
TMA/UMMA layouts, K grouping and the fused epilogue independently of rounding.
Accuracy: the error against the oracle, relative to S (sum of |terms|), is
reported per mode and bounded by the unit roundoff of the operands.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu

TC = ("bf16", "bf16x3", "tf32")
ALL = ("fp64", "fp32") + TC
# max |err| / S allowed per mode: 2 operand roundings of the mode's unit
# roundoff (bf16 2^-9, tf32 2^-11, split bf16 ~2^-17) plus FP32 accumulation
BOUND = {"bf16": 2 ** -7, "tf32": 2 ** -9, "bf16x3": 2 ** -13}


def run(tab, F, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    O = fk.conv(tab, torch.tensor(F, dtype=dt, device="cuda"), prec)
    torch.cuda.synchronize()
    assert fk._lib.load().fk_device_status(1) == 0
    return O.double().cpu().numpy()


def int_table(seed, nd, nc, nx, nxg, R, lo=-3, hi=4):
    rng = np.random.default_rng(seed)
    ca, cb = W.channels(rng, nc)
    t = W.HadTable(rng.integers(lo, hi, (nd, nc, nx, nx)).astype(np.float64), ca, cb,
                   np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32), nxg)
    F = rng.integers(lo, hi, (R, 14, nxg)).astype(np.float64)
    return t, F


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("shape", [(5, 6, 5, 9, 3), (37, 20, 17, 20, 130), (9, 196, 3, 3, 1),
                                   (13, 3, 33, 40, 129), (4, 11, 64, 64, 257), (1, 1, 1, 1, 1)])
def test_tc_exact_small_integers(prec, shape):
    nd, nc, nx, nxg, R = shape
    t, F = int_table(sum(shape), nd, nc, nx, nxg, R)
    O_ref, _ = oracle.had(t, F)
    tab = fk.Table.from_workload(t, precs=(prec,))
    O = run(tab, F, prec)
    assert np.array_equal(O, O_ref), np.abs(O - O_ref).max()


@pytest.mark.parametrize("R", [100, 512])
def test_tc_config_errors(R):
    """Configs 1 and 2: error per mode against the FP64 oracle."""
    t, F = W.config1(R=R) if R == 100 else W.config2(R=R)
    O_ref, S = oracle.had(t, F)
    tab = fk.Table.from_workload(t, precs=ALL)
    report = {}
    for prec in TC:
        O = run(tab, F, prec)
        e = np.abs(O - O_ref)
        report[prec] = (float((e / S).max()), float(np.median(e / np.abs(O_ref))))
        assert (e / S).max() <= BOUND[prec], (prec, report[prec])
    print("max err/S, median err/|O|:", report)
    # the split operands must win back accuracy over plain BF16
    assert report["bf16x3"][0] < report["bf16"][0] / 50


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (129, 3, 17, 5), (65, 13, 64, 66), (200, 60, 30, 257),
                                   (7, 196, 3, 128), (33, 14, 50, 1)])
def test_tc_ragged(prec, shape):
    nd, nc, nx, R = shape
    rng = np.random.default_rng(nd + nc + nx + R)
    x = W.xgrid(nx, 1e-6)
    t = W.had_table(rng, nd, nc, x)
    F = W.pdf_replicas(x, W.pdf_params(rng), R, rng)
    O_ref, S = oracle.had(t, F)
    tab = fk.Table.from_workload(t, precs=(prec,))
    O = run(tab, F, prec)
    assert (np.abs(O - O_ref) / S).max() <= BOUND[prec]


@pytest.mark.parametrize("prec", TC)
def test_tc_replica_independent_of_batch(prec):
    t, F = W.config1(R=300)
    tab = fk.Table.from_workload(t, precs=(prec,))
    full = run(tab, F, prec)
    part = run(tab, F[37:37 + 64], prec)
    one = run(tab, F[200:201], prec)
    assert np.array_equal(full[37:37 + 64], part)
    assert np.array_equal(full[200:201], one)


@pytest.mark.parametrize("prec", TC)
def test_tc_pair_launch_matches_single(prec):
    """An even number of replica tiles runs on CTA pairs (256-row MMAs over two
    SMs), an odd number on single CTAs: every replica's result is bit-identical."""
    t, F = W.config1(R=1024)
    tab = fk.Table.from_workload(t, precs=(prec,))
    pair = run(tab, F, prec)               # 8 replica tiles: pairs
    single = run(tab, F[128:512], prec)    # 3 replica tiles: single CTAs
    assert np.array_equal(pair[128:512], single)
    O_ref, S = oracle.had(t, F[:64])
    assert (np.abs(pair[:64] - O_ref) / S).max() <= BOUND[prec]
    gO = np.random.default_rng(5).standard_normal((1024, t.fk.shape[0]))
    g_pair = run_bwd(tab, F[:256], gO[:256], prec)
    g_single = run_bwd(tab, F[:128], gO[:128], prec)
    assert np.array_equal(g_pair[:128], g_single)


def test_tc_shared_grid_and_ldo():
    """Tables on subsets of a master grid, written into one wide output."""
    g = W.config3(R=130, scale=0.05)
    had = [t for t in g.tables if hasattr(t, "ca")][:5]
    ntot = sum(t.ndata for t in had)
    out = torch.full((130, ntot + 3), float("nan"), device="cuda")
    Fd = torch.tensor(g.F, dtype=torch.float32, device="cuda")
    off = 0
    refs = []
    for t in had:
        tab = fk.Table.from_workload(t, precs=("bf16x3",))
        fk.conv(tab, Fd, "bf16x3", out=out[:, off:off + t.ndata])
        refs.append(oracle.had(t, g.F))
        off += t.ndata
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    off = 0
    for t, (O_ref, S) in zip(had, refs):
        assert (np.abs(got[:, off:off + t.ndata] - O_ref) / S).max() <= BOUND["bf16x3"]
        off += t.ndata
    assert np.isnan(got[:, ntot:]).all()


# ------------------------------------------------------------ adjoint ----

def _grad_scale(t, F, gO):
    a = W.HadTable(np.abs(t.fk), t.ca, t.cb, t.xmap, t.nxg)
    return oracle.had_grad(a, np.abs(F), np.abs(gO))


def run_bwd(tab, F, gO, prec, gF=None, accumulate=False):
    out = fk.conv_backward(tab, torch.tensor(F, dtype=torch.float32, device="cuda"),
                           torch.tensor(gO, dtype=torch.float32, device="cuda"), prec,
                           gF=gF, accumulate=accumulate)
    torch.cuda.synchronize()
    assert fk._lib.load().fk_device_status(1) == 0
    return out.double().cpu().numpy()


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("shape", [(5, 6, 5, 9, 3), (37, 20, 17, 20, 130), (13, 3, 33, 40, 129),
                                   (4, 11, 64, 64, 2), (1, 1, 1, 1, 1), (9, 196, 3, 3, 5)])
def test_tc_adjoint_exact_small_integers(prec, shape):
    nd, nc, nx, nxg, R = shape
    t, F = int_table(sum(shape) + 1, nd, nc, nx, nxg, R)
    gO = np.random.default_rng(9).integers(-3, 4, (R, nd)).astype(np.float64)
    ref = oracle.had_grad(t, F, gO)
    tab = fk.Table.from_workload(t, precs=(prec,))
    assert np.array_equal(run_bwd(tab, F, gO, prec), ref)


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("shape", [(200, 60, 30, 100), (129, 13, 50, 7), (33, 196, 8, 200), (7, 2, 17, 1)])
def test_tc_adjoint_accuracy(prec, shape):
    nd, nc, nx, R = shape
    rng = np.random.default_rng(sum(shape))
    x = W.xgrid(nx, 1e-6)
    t = W.had_table(rng, nd, nc, x)
    F = W.pdf_replicas(x, W.pdf_params(rng), R, rng)
    gO = rng.standard_normal((R, nd))
    ref = oracle.had_grad(t, F, gO)
    S = _grad_scale(t, F, gO)
    tab = fk.Table.from_workload(t, precs=(prec,))
    got = run_bwd(tab, F, gO, prec)
    err = (np.abs(got - ref) / np.maximum(S, 1e-300)).max()
    print(prec, shape, "adjoint max err/S", err)
    assert err <= BOUND[prec]


def test_tc_adjoint_accumulates():
    g = W.config3(R=9, scale=0.05)
    had = [t for t in g.tables if hasattr(t, "ca")][:4]
    gF = torch.zeros(g.F.shape, dtype=torch.float32, device="cuda")
    ref = np.zeros_like(g.F)
    S = np.zeros_like(g.F)
    rng = np.random.default_rng(4)
    for t in had:
        gO = rng.standard_normal((9, t.ndata))
        ref += oracle.had_grad(t, g.F, gO)
        S += _grad_scale(t, g.F, gO)
        tab = fk.Table.from_workload(t, precs=("bf16x3",))
        run_bwd(tab, g.F, gO, "bf16x3", gF=gF, accumulate=True)
    got = gF.double().cpu().numpy()
    assert (np.abs(got - ref) / np.maximum(S, 1e-300)).max() <= BOUND["bf16x3"]
