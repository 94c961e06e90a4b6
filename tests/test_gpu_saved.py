"""Saved forward products (fk_had_conv_save / fk_conv_backward_saved).

The adjoint's derivative with respect to the first flavour of each channel
(the gradient of Eq. 1 that every fit step needs, Sec. 2) is the forward's
tensor-core product Y_g contracted with gO instead of f_{a_g}.  The saving
forward must give the same O bit for bit, and the saved adjoint the same gF
bit for bit as fk_conv_backward (its contraction runs in the order of the
adjoint's epilogue); both are also pinned to the FP64 oracle: exactly on
small-integer tables, within the mode's bound on realistic ones.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu

TC = ("bf16", "bf16x3", "tf32")
# the bounds of the tensor-core adjoint (max |err| / S, S = sum of |terms|)
BOUND = {"bf16": 2 ** -7, "tf32": 2 ** -9, "bf16x3": 3 * 2 ** -16}


def int_table(seed, nd, nc, nx, nxg, R):
    rng = np.random.default_rng(seed)
    ca, cb = W.channels(rng, nc)
    t = W.HadTable(rng.integers(-3, 4, (nd, nc, nx, nx)).astype(np.float64), ca, cb,
                   np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32), nxg)
    F = rng.integers(-3, 4, (R, 14, nxg)).astype(np.float64)
    gO = rng.integers(-3, 4, (R, nd)).astype(np.float64)
    return t, F, gO


def both(tab, F, gO, prec, ldo=0, accumulate=False, gF0=None):
    """(O, gF) of the plain calls and of the saved-product calls, on device."""
    R = F.shape[0]
    Fd = torch.tensor(F, dtype=torch.float32, device="cuda")
    wide = tab.ndata + ldo
    gOw = torch.full((R, wide), float("nan"), device="cuda")
    gOw[:, :tab.ndata] = torch.tensor(gO, dtype=torch.float32, device="cuda")
    gOd = gOw[:, :tab.ndata]
    out = []
    # NaN everywhere first: a product read that the forward did not write
    # would reach gF
    sv = fk.saved_buffer(tab, R, prec).fill_(float("nan"))
    for saved in (None, sv):
        Ow = torch.full((R, wide), float("nan"), device="cuda")
        O = fk.conv(tab, Fd, prec, out=Ow[:, :tab.ndata], save=saved)
        gF = (gF0.clone() if gF0 is not None else torch.full((R, 14, tab.nxg), float("nan"), device="cuda"))
        fk.conv_backward(tab, Fd, gOd, prec, gF=gF, accumulate=accumulate, saved=saved)
        torch.cuda.synchronize()
        assert fk._lib.load().fk_device_status(1) == 0
        assert torch.isnan(Ow[:, tab.ndata:]).all()
        out.append((O.double().cpu().numpy(), gF.double().cpu().numpy()))
    return out


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("shape", [(5, 6, 5, 9, 3), (37, 20, 17, 20, 130), (13, 3, 33, 40, 129),
                                   (4, 11, 64, 64, 2), (1, 1, 1, 1, 1), (9, 196, 3, 3, 5), (20, 30, 12, 16, 256)])
def test_saved_exact_small_integers(prec, shape):
    nd, nc, nx, nxg, R = shape
    t, F, gO = int_table(sum(shape) + 7, nd, nc, nx, nxg, R)
    O_ref, _ = oracle.had(t, F)
    g_ref = oracle.had_grad(t, F, gO)
    tab = fk.Table.from_workload(t, precs=(prec,))
    (O0, g0), (O1, g1) = both(tab, F, gO, prec)
    assert np.array_equal(O1, O_ref) and np.array_equal(O0, O_ref)
    assert np.array_equal(g1, g_ref), np.abs(g1 - g_ref).max()
    assert np.array_equal(g0, g_ref)


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("shape", [(200, 60, 30, 100), (129, 13, 50, 7), (33, 196, 8, 200), (7, 2, 17, 1),
                                   (90, 40, 41, 256), (300, 25, 44, 130)])
def test_saved_bitwise_and_accuracy(prec, shape):
    nd, nc, nx, R = shape
    rng = np.random.default_rng(sum(shape) + 3)
    x = W.xgrid(nx, 1e-6)
    t = W.had_table(rng, nd, nc, x)
    F = W.pdf_replicas(x, W.pdf_params(rng), R, rng)
    gO = rng.standard_normal((R, nd))
    tab = fk.Table.from_workload(t, precs=(prec,))
    (O0, g0), (O1, g1) = both(tab, F, gO, prec, ldo=3)
    assert np.array_equal(O0, O1)
    assert np.array_equal(g0, g1), np.abs(g0 - g1).max()
    ref = oracle.had_grad(t, F, gO)
    a = W.HadTable(np.abs(t.fk), t.ca, t.cb, t.xmap, t.nxg)
    S = oracle.had_grad(a, np.abs(F), np.abs(gO))
    err = (np.abs(g1 - ref) / np.maximum(S, 1e-300)).max()
    print(prec, shape, "saved adjoint max err/S", err)
    assert err <= BOUND[prec]


def test_saved_accumulates():
    rng = np.random.default_rng(11)
    x = W.xgrid(25, 1e-6)
    t = W.had_table(rng, 40, 30, x)
    F = W.pdf_replicas(x, W.pdf_params(rng), 17, rng)
    gO = rng.standard_normal((17, 40))
    tab = fk.Table.from_workload(t, precs=("bf16x3",))
    gF0 = torch.tensor(rng.standard_normal((17, 14, t.nxg)), dtype=torch.float32, device="cuda")
    (_, g0), (_, g1) = both(tab, F, gO, "bf16x3", accumulate=True, gF0=gF0)
    assert np.array_equal(g0, g1)
    plain = fk.conv_backward(tab, torch.tensor(F, dtype=torch.float32, device="cuda"),
                             torch.tensor(gO, dtype=torch.float32, device="cuda"), "bf16x3")
    assert np.array_equal(g1, (gF0 + plain).double().cpu().numpy())


def test_saved_size_and_errors():
    rng = np.random.default_rng(5)
    x = W.xgrid(20, 1e-6)
    t = W.had_table(rng, 50, 12, x)
    tab = fk.Table.from_workload(t, precs=("bf16x3", "fp32"))
    F = torch.tensor(W.pdf_replicas(x, W.pdf_params(rng), 3, rng), dtype=torch.float32, device="cuda")
    n1, n128, n129 = (fk.saved_size(tab, R, "bf16x3") for R in (1, 128, 129))
    assert n1 == n128 and n129 == 2 * n128
    # at least the products themselves: 4 bytes x ndata x groups x nx x 128
    groups = len(set(np.asarray(t.ca).tolist()))
    assert n1 >= 4 * 50 * groups * 20 * 128
    buf = fk.saved_buffer(tab, 3, "bf16x3")
    with pytest.raises(fk.FKError) as e:
        fk.conv(tab, F, "bf16x3", save=buf[:-1])
    assert e.value.status == fk._lib.FK_EINVAL and "needed" in str(e.value)
    with pytest.raises(fk.FKError) as e:
        fk.saved_size(tab, 3, "fp32")
    assert e.value.status == fk._lib.FK_EUNSUPPORTED
    with pytest.raises(fk.FKError) as e:
        fk.saved_size(tab, 3, "tf32")  # not stored
    assert e.value.status == fk._lib.FK_EUNSUPPORTED
    with pytest.raises(fk.FKError) as e:
        fk.saved_size(tab, 0, "bf16x3")
    assert e.value.status == fk._lib.FK_EINVAL
    lum = fk.Table.from_workload(t, precs=("bf16x3",), form="lumi")
    with pytest.raises(fk.FKError) as e:
        fk.saved_size(lum, 3, "bf16x3")
    assert e.value.status == fk._lib.FK_EUNSUPPORTED
    d = W.dis_table(rng, 30, 5, x)
    dtab = fk.Table.from_workload(d, precs=("bf16x3",))
    with pytest.raises(fk.FKError) as e:
        fk.saved_size(dtab, 3, "bf16x3")
    assert e.value.status == fk._lib.FK_EINVAL
    assert fk._lib.load().fk_device_status(1) == 0
