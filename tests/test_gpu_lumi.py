"""The hadronic forward in the paper's dense formulation (Sec. 3, Table 3)
with the PDF matrix L[r][(c, i, j)] = f_{a_c}(x_i) f_{b_c}(x_j) formed in
shared memory (FK_TABLE_LUMI), against the FP64 oracle.

Pins: small-integer tables and PDFs are exact in every reduced mode (the
flattened packing, the builders' gather of f values, the swizzled layout of
the built operand, the K splits and their fixed-order sum); split-BF16
operands with lo parts on either flavour or on the table are exact in BF16X3
and not in BF16 (both cross terms of the built operand); on the
configuration tables every mode stays within its bound of S = sum |terms|;
the result of a replica does not depend on R (the K split is a table
property); the dense and the factorised forms agree within the bound; the
factorised form is the default and the dense form is taken on request only.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu

TC = ("bf16", "bf16x3", "tf32")
# per-product bounds of the modes (two roundings of the built operand's
# product and of the table value; tests/test_gpu_tc.py) plus the FP32
# accumulation of one K split (1536 products) and of the partial tiles,
# at most 1600 * 2^-24 of S
BOUND = {"bf16": 2 ** -7, "tf32": 2 ** -9, "bf16x3": 3 * 2 ** -16}
ACC = 1600 * 2.0 ** -24


def fwd(tab, F, prec):
    O = fk.conv(tab, torch.tensor(F, dtype=torch.float32, device="cuda"), prec)
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


# (ndata, channels, nx, grid, R): several K splits (K = nc nx nxp > 1536),
# nx not a multiple of 8 (padded columns), nx = 1, one channel, more than one
# data tile (ndata > 256), paired and odd replica tiles, R = 1
SHAPES = [(37, 20, 17, 20, 130), (300, 9, 11, 16, 257), (5, 1, 1, 1, 1), (64, 196, 3, 5, 3),
          (200, 12, 30, 30, 128), (17, 40, 8, 9, 2)]


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("shape", SHAPES)
def test_lumi_exact_small_integers(prec, shape):
    nd, nc, nx, nxg, R = shape
    t, F = int_table(sum(shape), nd, nc, nx, nxg, R, lo=-2, hi=3)
    tab = fk.Table.from_workload(t, precs=(prec,), form="lumi")
    assert tab.lumi
    O_ref, _ = oracle.had(t, F)
    O = fwd(tab, F, prec)
    assert np.array_equal(O, O_ref), np.abs(O - O_ref).max()


def split_values(rng, shape):
    h = rng.integers(1, 3, shape) * rng.choice([-1.0, 1.0], shape)
    return h + rng.integers(-3, 4, shape) * 2.0 ** -10


@pytest.mark.parametrize("side", ["F_b", "F_a", "FK"])
def test_lumi_bf16x3_cross_terms_exact(side):
    """Channels (a, b) with a in 0..6 and b in 7..13; the flavours of one side
    carry values h + l (h = +-1, +-2, l = k 2^-10), the others -1..1 (powers of
    two or zero).  Each product f_a f_b is then 2^e (h + l) or zero, held
    exactly as hi + lo, and with |FK| <= 1 every FP32 partial sum is a
    multiple of 2^-10 below 2^14: BF16X3 must equal the oracle bit for bit,
    plain BF16 must not."""
    rng = np.random.default_rng(11 + len(side))
    nd, nx, nxg, R = 40, 9, 12, 130
    pairs = [(a, b) for a in range(7) for b in range(7, 14)]
    sel = rng.choice(len(pairs), 6, replace=False)
    ca = np.array([pairs[k][0] for k in sel], np.int32)
    cb = np.array([pairs[k][1] for k in sel], np.int32)
    shape = (nd, 6, nx, nx)
    fkv = split_values(rng, shape) / 2 if side == "FK" else rng.integers(-1, 2, shape).astype(np.float64)
    t = W.HadTable(fkv, ca, cb, np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32), nxg)
    F = rng.integers(-1, 2, (R, 14, nxg)).astype(np.float64)
    if side == "F_b":
        F[:, 7:] = split_values(rng, (R, 7, nxg))
    elif side == "F_a":
        F[:, :7] = split_values(rng, (R, 7, nxg))
    tab = fk.Table.from_workload(t, precs=("bf16x3", "bf16"), form="lumi")
    O_ref, _ = oracle.had(t, F)
    assert np.array_equal(fwd(tab, F, "bf16x3"), O_ref)
    assert not np.array_equal(fwd(tab, F, "bf16"), O_ref)


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("R", [100, 512])
def test_lumi_config_accuracy(prec, R):
    """Config 1 (R = 100) and config 2 (R = 512) shaped table: error against
    the FP64 oracle within the mode's bound of S; the factorised form of the
    same table agrees within twice the bound."""
    t, _ = W.config1(R=1)
    rng = np.random.default_rng(R)
    F = W.pdf_replicas(W.xgrid(30, 1e-6), W.pdf_params(rng), R, rng)
    O_ref, S = oracle.had(t, F)
    lum = fk.Table.from_workload(t, precs=(prec,), form="lumi")
    assert lum.lumi
    fac = fk.Table.from_workload(t, precs=(prec,))
    assert not fk.Table.from_workload(t, precs=(prec,), form="factored").lumi
    assert not fac.lumi
    e_l = float((np.abs(fwd(lum, F, prec) - O_ref) / S).max())
    e_f = float((np.abs(fwd(fac, F, prec) - O_ref) / S).max())
    print(prec, R, "max err/S dense", e_l, "factorised", e_f)
    assert e_l <= BOUND[prec] + ACC
    assert float((np.abs(fwd(lum, F, prec) - fwd(fac, F, prec)) / S).max()) <= 2 * (BOUND[prec] + ACC)


@pytest.mark.parametrize("prec", TC)
def test_lumi_replica_independent_of_R(prec):
    t, F = int_table(5, 120, 24, 20, 25, 300, lo=-50, hi=50)
    F = F * 0.0137  # non-integer values: results round, the order must not change
    tab = fk.Table.from_workload(t, precs=(prec,), form="lumi")
    full = fwd(tab, F, prec)
    assert np.array_equal(full[37:37 + 64], fwd(tab, F[37:37 + 64], prec))
    assert np.array_equal(full[299:300], fwd(tab, F[299:300], prec))
    assert np.array_equal(full[:256], fwd(tab, F[:256], prec))


def test_lumi_ldo_and_adjoint_unchanged():
    """Outputs land at their row stride and leave the rest alone; the adjoint
    of a dense-form table (factorised in both cases) equals the factorised
    table's bit for bit."""
    t, F = int_table(9, 70, 30, 12, 14, 40)
    lum = fk.Table.from_workload(t, precs=("bf16x3",), form="lumi")
    fac = fk.Table.from_workload(t, precs=("bf16x3",), form="factored")
    Fd = torch.tensor(F, dtype=torch.float32, device="cuda")
    out = torch.full((40, 70 + 5), float("nan"), device="cuda")
    fk.conv(lum, Fd, "bf16x3", out=out[:, 2:72])
    torch.cuda.synchronize()
    O_ref, _ = oracle.had(t, F)
    o = out.double().cpu().numpy()
    assert np.array_equal(o[:, 2:72], O_ref)
    assert np.isnan(o[:, :2]).all() and np.isnan(o[:, 72:]).all()
    gO = torch.tensor(np.random.default_rng(2).integers(-2, 3, (40, 70)), dtype=torch.float32, device="cuda")
    g1 = fk.conv_backward(lum, Fd, gO, "bf16x3")
    g2 = fk.conv_backward(fac, Fd, gO, "bf16x3")
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)


def test_lumi_is_opt_in():
    """The factorised form is the default for every table; the dense form
    only on request."""
    t1, _ = W.config1(R=1)
    assert not fk.Table.from_workload(t1, precs=("bf16",)).lumi
    small, _ = int_table(1, 10, 30, 30, 30, 1)
    assert not fk.Table.from_workload(small, precs=("bf16",)).lumi
    assert fk.Table.from_workload(small, precs=("bf16",), form="lumi").lumi


def test_lumi_served_alone_equals_mixed():
    """A dense-form table in the serving loop: a request's result is the same
    alone and coalesced with others (the K split does not depend on R)."""
    t, F = int_table(21, 150, 20, 20, 22, 64, lo=-40, hi=40)
    F = F * 0.011
    tab = fk.Table.from_workload(t, precs=("bf16x3",), form="lumi")
    srv = fk.Server(budget_bytes=8 << 30, max_inflight=1)
    tid = srv.add_table(tab)
    alone = srv.wait(srv.submit(tid, F[:10], "bf16x3"))
    tks = [srv.submit(tid, F[10 * k:10 * k + 10], "bf16x3") for k in range(6)]
    outs = [srv.wait(tk) for tk in tks]
    assert np.array_equal(outs[0], alone)
    O = fwd(tab, F[:60], "bf16x3")
    assert np.array_equal(np.concatenate(outs), O.astype(np.float32))
    srv.close()
