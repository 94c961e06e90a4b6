"""The dense product of the paper's timing study (Sec. 3, Table 3) on the GPU.

O[r][d] = sum_k FK[d][k] L[r][k] with the table flattened to [ndata][K] and
the PDF matrix L built per replica.  Pins: small-integer tables and PDF
matrices are exact in every mode (BF16/TF32 operands hold small integers
exactly and the FP32 sums stay below 2^24), across data and replica tiles and
ragged K; the PDF matrix kernel is exact against the oracle; on the Table 3
base table (49 channels, 27 x points, K = 35721) the product of the GPU PDF
matrix equals Eq. 1 (oracle) within each mode's bound.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import _lib
from paper_1909_10547_b300 import workloads as W

pytestmark = pytest.mark.gpu

ALL = ("fp64", "fp32", "bf16", "bf16x3", "tf32")
# max |err| / S per mode: FP64/FP32 as the other parity tests; the tensor-core
# modes as for Eq. 1 (two operand roundings of the mode plus FP32 sums)
BOUND = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 2 ** -7, "tf32": 2 ** -9, "bf16x3": 3 * 2 ** -16}


def _dt(prec):
    return torch.float64 if prec == "fp64" else torch.float32


def run_dense(tab, L, prec):
    O = fk.dense_conv(tab, torch.tensor(L, dtype=_dt(prec), device="cuda"), prec)
    torch.cuda.synchronize()
    assert _lib.load().fk_device_status(1) == 0
    return O.double().cpu().numpy()


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 37, 3), (17, 100, 130), (300, 1000, 257),
                                   (257, 35, 129), (40, 4099, 2), (8, 35721, 100), (3, 20000, 1)])
def test_dense_exact_small_integers(shape):
    """(ndata, K, R): ragged K (not a multiple of the K step or the stage),
    two data tiles (300 > 256), paired (R = 130) and odd (257, 129) replica
    tile counts; few tiles with long K (the last three) take the K split of
    the tensor-core path, whose last split runs past K on zero-filled
    operands."""
    nd, K, R = shape
    rng = np.random.default_rng(nd * 7 + K + R)
    fkd = rng.integers(-4, 5, (nd, K)).astype(np.float64)
    L = rng.integers(-4, 5, (R, K)).astype(np.float64)
    O_ref, _ = oracle.dense(fkd, L)
    tab = fk.Table.dense(fkd, precs=ALL)
    for prec in ALL:
        O = run_dense(tab, L, prec)
        assert np.array_equal(O, O_ref), (prec, np.abs(O - O_ref).max())


@pytest.mark.parametrize("side", ["L", "FK"])
@pytest.mark.parametrize("shape", [(5, 37, 3), (300, 1000, 130), (8, 4099, 1)])
def test_dense_bf16x3_cross_terms_exact(side, shape):
    """Split operands in the dense product: one side holds v = h + l (h = +-1,
    +-2 and l = k 2^-10, |k| <= 3: hi = h and lo = l exactly), the other side
    integers in -1..1, so hi*hi + hi*lo + lo*hi is the exact product and the
    FP32 sums (multiples of 2^-10, below 2^14) are exact: bit-equal to the
    oracle.  Plain BF16 drops the lo parts and differs."""
    nd, K, R = shape
    rng = np.random.default_rng(nd + K + R + len(side))

    def split(shape_):
        h = rng.integers(1, 3, shape_) * rng.choice([-1.0, 1.0], shape_)
        return h + rng.integers(-3, 4, shape_) * 2.0 ** -10

    ints = lambda shape_: rng.integers(-1, 2, shape_).astype(np.float64)  # noqa: E731
    fkd = split((nd, K)) if side == "FK" else ints((nd, K))
    L = split((R, K)) if side == "L" else ints((R, K))
    O_ref, _ = oracle.dense(fkd, L)
    tab = fk.Table.dense(fkd, precs=("bf16x3", "bf16"))
    assert np.array_equal(run_dense(tab, L, "bf16x3"), O_ref)
    assert not np.array_equal(run_dense(tab, L, "bf16"), O_ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_luminosity_is_exact(prec):
    t, F = W.table3(4, 5)
    tab = fk.Table.from_workload(t, precs=(prec,))
    L = fk.luminosity(tab, torch.tensor(F, dtype=_dt(prec), device="cuda"), prec)
    torch.cuda.synchronize()
    got = L.double().cpu().numpy()
    if prec == "fp64":
        want = oracle.luminosity(t, F)
    else:  # one FP32 rounding of the product of the FP32 inputs
        F32 = F.astype(np.float32)
        want = oracle.luminosity(t, F32.astype(np.float64)).astype(np.float32).astype(np.float64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("R", [1, 3, 100])
def test_dense_table3_matches_eq1(R):
    """The paper's base table at ndata = 64: dense product of the GPU PDF
    matrix against Eq. 1 from the oracle, every mode within its bound."""
    t, F = W.table3(64, R)
    O_ref, S = oracle.had(t, F)
    ht = fk.Table.from_workload(t, precs=("fp64", "fp32"))
    tab = fk.Table.dense(t.fk.reshape(t.fk.shape[0], -1), precs=ALL)
    report = {}
    for prec in ALL:
        Fd = torch.tensor(F, dtype=_dt("fp64" if prec == "fp64" else "fp32"), device="cuda")
        L = fk.luminosity(ht, Fd, "fp64" if prec == "fp64" else "fp32")
        O = fk.dense_conv(tab, L, prec)
        torch.cuda.synchronize()
        assert _lib.load().fk_device_status(1) == 0
        err = float((np.abs(O.double().cpu().numpy() - O_ref) / S).max())
        report[prec] = err
        assert err <= BOUND[prec], (prec, err)
    print("max err/S:", report)


def test_dense_rejects_other_calls():
    rng = np.random.default_rng(3)
    tab = fk.Table.dense(rng.standard_normal((4, 50)), precs=("fp32",))
    L = torch.zeros((2, 50), dtype=torch.float32, device="cuda")
    O = torch.empty((2, 4), dtype=torch.float32, device="cuda")
    lib = _lib.load()
    stream = fk._stream()
    assert lib.fk_had_conv(tab.handle, fk._p(L), 2, fk._p(O), 0, _lib.FK_FP32, stream) == _lib.FK_EINVAL
    assert lib.fk_conv_backward(tab.handle, fk._p(L), fk._p(O), 0, 2, fk._p(L), 0, _lib.FK_FP32,
                                stream) == _lib.FK_EUNSUPPORTED
    # a mode the table does not hold
    assert lib.fk_dense_conv(tab.handle, fk._p(L), 2, fk._p(O), 0, _lib.FK_BF16, stream) == _lib.FK_EUNSUPPORTED
    with pytest.raises(ValueError):
        fk.dense_conv(tab, torch.zeros((2, 49), dtype=torch.float32, device="cuda"), "fp32")
