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
# roundoff (BF16, 8 significant bits: 2^-8; TF32, 11 bits: 2^-11) plus FP32
# accumulation.  Split BF16 holds each operand to 2^-16 of its value
# (hi = bf16(v), lo = bf16(v - hi): two 8-bit roundings) and drops lo*lo (at
# most 2^-16 of the product), so a single product is within 3 * 2^-16 of
# exact: the bound of the few-term shapes (measured at most 1.6e-5 = 2^-16).
# Over many terms the errors average out: on the configuration tables (54 000
# terms per point) the bound is 2^-20 (measured 2.4e-7 to 2.9e-7).
BOUND = {"bf16": 2 ** -7, "tf32": 2 ** -9, "bf16x3": 3 * 2 ** -16}
BOUND_CONFIG = {"bf16": 2 ** -9, "tf32": 2 ** -11, "bf16x3": 2 ** -20}


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


# ---------------------------------------------- split-operand (hi + lo) pins
# Values v = h + l with h = +-1 or +-2 and l = k * 2^-10, |k| <= 3: bf16(v) = h
# exactly (|l| is below half a BF16 unit of h) and v - h = l is exact in BF16,
# so BF16X3 holds v as hi = h, lo = l.  When only one operand of a product
# carries a lo part, hi*hi + hi*lo + lo*hi is the exact product (the dropped
# lo*lo is zero).  With |FK| <= 1, |F| <= 2.003, |gO| <= 2 and 6 channels every
# FP32 partial sum is a multiple of 2^-10 below 2^14 in magnitude, hence exact,
# so the result must equal the FP64 oracle bit for bit.  Dropping either cross
# term, or pairing a lo copy with the wrong operand, moves it by multiples of
# 2^-10.

def split_values(rng, shape):
    h = rng.integers(1, 3, shape) * rng.choice([-1.0, 1.0], shape)
    return h + rng.integers(-3, 4, shape) * 2.0 ** -10


def split_table(seed, nd, nx, nxg, R, side):
    """Channels (a, b) with a in 0..6 and b in 7..13.  side = "F_b": the
    second flavour's PDF values carry lo parts (the forward MMA operand and
    the adjoint's first term); "F_a": the first flavour's (the adjoint's second
    term, the transposed packing's MMA operand); "FK": the table carries them."""
    rng = np.random.default_rng(seed)
    pairs = [(a, b) for a in range(7) for b in range(7, 14)]
    sel = rng.choice(len(pairs), 6, replace=False)
    ca = np.array([pairs[k][0] for k in sel], np.int32)
    cb = np.array([pairs[k][1] for k in sel], np.int32)
    shape = (nd, len(ca), nx, nx)
    fkv = split_values(rng, shape) / 2 if side == "FK" else rng.integers(-1, 2, shape).astype(np.float64)
    t = W.HadTable(fkv, ca, cb, np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32), nxg)
    F = rng.integers(-2, 3, (R, 14, nxg)).astype(np.float64)
    if side == "F_b":
        F[:, 7:] = split_values(rng, (R, 7, nxg))
    elif side == "F_a":
        F[:, :7] = split_values(rng, (R, 7, nxg))
    return t, F


@pytest.mark.parametrize("side", ["F_b", "F_a", "FK"])
@pytest.mark.parametrize("shape", [(5, 4, 9, 3), (37, 7, 20, 130), (9, 3, 3, 257)])
def test_bf16x3_cross_terms_exact(side, shape):
    nd, nx, nxg, R = shape
    t, F = split_table(sum(shape) + len(side), nd, nx, nxg, R, side)
    tab = fk.Table.from_workload(t, precs=("bf16x3", "bf16"))
    O_ref, _ = oracle.had(t, F)
    O = run(tab, F, "bf16x3")
    assert np.array_equal(O, O_ref), np.abs(O - O_ref).max()
    gO = np.random.default_rng(3).integers(-2, 3, (R, nd)).astype(np.float64)
    g_ref = oracle.had_grad(t, F, gO)
    assert np.array_equal(run_bwd(tab, F, gO, "bf16x3"), g_ref)
    # the same inputs through plain BF16 lose the lo parts: the pin has teeth
    # (with lo parts on the first flavour only the adjoint's MMA sees them; the
    # forward applies that flavour in FP32 in its epilogue)
    if side != "F_a":
        assert not np.array_equal(run(tab, F, "bf16"), O_ref)
    assert not np.array_equal(run_bwd(tab, F, gO, "bf16"), g_ref)


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
        assert (e / S).max() <= BOUND_CONFIG[prec], (prec, report[prec])
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
    err = (np.abs(O - O_ref) / S).max()
    print(prec, shape, "forward max err/S", err)
    assert err <= BOUND[prec]


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
