"""FP64 results on the tensor cores (FK_FP64_TC: exact BF16 digit slices).

Each FP64 operand is cut into 8 digits of 7 bits per row and K chunk; the 36
leading digit products run as BF16 MMAs with exact FP32 sums and are added in
FP64.  Pins: small integers are exact (bit-equal to the FP64 oracle) for the
dense product, DIS and hadronic tables, forward and adjoint; against the
oracle every result meets the FP64 contract, 1e-12 of S = sum |terms|, on
the configuration tables (config 0 DIS, config 1 hadronic, the DIS and
hadronic tables of the global set, Table 3's base table); with values spread
over 60 orders of magnitude in a row the error stays within the scheme's own
bound (per K chunk of 512, 2^-48 K_c times the rows' largest values); a replica's
result does not depend on R; the fit step in this mode matches the oracle
chain at 1e-12.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import workloads as W
from paper_1909_10547_b300.fitstep import GlobalFit

from bounds import fit_chain_scales

pytestmark = pytest.mark.gpu

P = "fp64tc"


def fwd(tab, F):
    O = fk.conv(tab, torch.tensor(F, device="cuda"), P)
    torch.cuda.synchronize()
    assert fk._lib.load().fk_device_status(1) == 0
    return O.cpu().numpy()


def bwd(tab, F, gO):
    g = fk.conv_backward(tab, torch.tensor(F, device="cuda"), torch.tensor(gO, device="cuda"), P)
    torch.cuda.synchronize()
    return g.cpu().numpy()


def abs_table(t):
    if hasattr(t, "ca"):
        return W.HadTable(np.abs(t.fk), t.ca, t.cb, t.xmap, t.nxg)
    return W.DisTable(np.abs(t.fk), t.flav, t.xmap, t.nxg)


@pytest.mark.parametrize("shape", [(1, 1, 1), (37, 1000, 130), (300, 2100, 3), (8, 4099, 257)])
def test_dense_exact_small_integers(shape):
    """(ndata, K, R): K over several 512 chunks (ragged last chunk), two data
    tiles, paired and odd replica tiles."""
    nd, K, R = shape
    rng = np.random.default_rng(sum(shape))
    fkd = rng.integers(-40, 41, (nd, K)).astype(np.float64)
    L = rng.integers(-40, 41, (R, K)).astype(np.float64)
    O_ref, _ = oracle.dense(fkd, L)
    tab = fk.Table.dense(fkd, precs=(P,))
    O = fk.dense_conv(tab, torch.tensor(L, device="cuda"), P)
    torch.cuda.synchronize()
    assert np.array_equal(O.cpu().numpy(), O_ref)


@pytest.mark.parametrize("kind", ["dis", "had"])
def test_exact_small_integers_forward_and_adjoint(kind):
    rng = np.random.default_rng(3 if kind == "dis" else 4)
    nd, nx, nxg, R = 45, 9, 12, 130
    xmap = np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32)
    if kind == "dis":
        flav = np.sort(rng.choice(14, 7, replace=False)).astype(np.int32)
        fkv = np.zeros((nd, 14, nx))
        fkv[:, flav, :] = rng.integers(-9, 10, (nd, 7, nx))
        t = W.DisTable(fkv, flav, xmap, nxg)
    else:
        ca, cb = W.channels(rng, 30)
        t = W.HadTable(rng.integers(-9, 10, (nd, 30, nx, nx)).astype(np.float64), ca, cb, xmap, nxg)
    F = rng.integers(-9, 10, (R, 14, nxg)).astype(np.float64)
    gO = rng.integers(-9, 10, (R, nd)).astype(np.float64)
    tab = fk.Table.from_workload(t, precs=(P,))
    assert np.array_equal(fwd(tab, F), oracle.conv(t, F)[0])
    assert np.array_equal(bwd(tab, F, gO), oracle.conv_grad(t, F, gO))


def _cases():
    t0, _ = W.config0()
    x0 = W.xgrid(40, 1e-7)
    rng = np.random.default_rng(5)
    yield "config 0 DIS, R=100", t0, W.pdf_replicas(x0, W.pdf_params(rng), 100, rng)
    t1, F1 = W.config1(R=100)
    yield "config 1 hadronic, R=100", t1, F1
    g = W.config3(R=20, scale=0.3)
    for t in g.tables[:6]:
        yield f"global-set {'hadronic' if hasattr(t, 'ca') else 'DIS'} table, ndata={t.ndata}", t, g.F


def test_fp64_contract_against_oracle():
    report = []
    for name, t, F in _cases():
        tab = fk.Table.from_workload(t, precs=(P,))
        O_ref, S = oracle.conv(t, F)
        err = float((np.abs(fwd(tab, F) - O_ref) / S).max())
        gO = np.random.default_rng(1).standard_normal((F.shape[0], t.ndata))
        g_ref = oracle.conv_grad(t, F, gO)
        scale = oracle.conv_grad(abs_table(t), np.abs(F), np.abs(gO))
        gerr = float((np.abs(bwd(tab, F, gO) - g_ref) / np.where(scale > 0, scale, 1.0)).max())
        report.append((name, err, gerr))
        assert err <= 1e-12 and gerr <= 1e-12, (name, err, gerr)
    print("FP64_TC max err/S (forward, adjoint):", report)


def test_table3_dense_against_oracle():
    t, F = W.table3(64, 20)
    Lm = oracle.luminosity(t, F)
    fk2 = t.fk.reshape(t.fk.shape[0], -1)
    O_ref, S = oracle.dense(fk2, Lm)
    tab = fk.Table.dense(fk2, precs=(P,))
    O = fk.dense_conv(tab, torch.tensor(Lm, device="cuda"), P).cpu().numpy()
    err = float((np.abs(O - O_ref) / S).max())
    print("Table 3 base table, FP64_TC max err/S", err)
    assert err <= 1e-12


def test_wide_dynamic_range_within_a_row():
    """Values over 60 orders of magnitude in one row.  The slices hold each
    value to within 2^-55 of the largest |value| of its row in its K chunk
    (chunks of 512), and each of the 28 dropped digit products is below
    2^-56 of the chunk's largest one, so per chunk the error is below
    K_c 2^-48 max|A_r| max|B_d|: the bound checked here.  (Relative to S this
    input is far outside the contract's reach: its largest elements of A and
    B never meet in one product.)"""
    rng = np.random.default_rng(9)
    nd, K, R = 20, 3000, 5
    fkd = rng.standard_normal((nd, K)) * 10.0 ** rng.uniform(-30, 30, (nd, K))
    L = rng.standard_normal((R, K)) * 10.0 ** rng.uniform(-30, 30, (R, K))
    O_ref, S = oracle.dense(fkd, L)
    tab = fk.Table.dense(fkd, precs=(P,))
    O = fk.dense_conv(tab, torch.tensor(L, device="cuda"), P).cpu().numpy()
    bound = np.zeros((R, nd))
    for c0 in range(0, K, 512):
        sl = slice(c0, min(K, c0 + 512))
        kc = sl.stop - sl.start
        bound += kc * 2.0 ** -48 * np.abs(L[:, sl]).max(axis=1)[:, None] * np.abs(fkd[:, sl]).max(axis=1)[None, :]
    assert np.all(np.abs(O - O_ref) <= bound)


def test_replica_independent_of_R():
    t, F = W.config1(R=300, ndata=60, nc=20, nx=20)
    tab = fk.Table.from_workload(t, precs=(P,))
    full = fwd(tab, F)
    assert np.array_equal(full[100:103], fwd(tab, F[100:103]))
    assert np.array_equal(full[299:300], fwd(tab, F[299:300]))


def test_fit_step_fp64_contract():
    """The whole fit step (forward, FP64 chi^2, adjoint) in FP64_TC against
    the oracle chain: 1e-12 of the componentwise scale and plain relative."""
    g = W.config3(R=6, scale=0.12, seed=77)
    o_true = [oracle.conv(t, g.F_true)[0][0] for t in g.tables]
    cov = W.covariance(o_true, 77)
    D = W.pseudo_data(o_true, 77)
    fit = GlobalFit(g.tables, g.F, cov.blocks, np.concatenate(D), prec=P)
    fit.step()
    torch.cuda.synchronize()
    chi_ref = np.zeros(6)
    gF_ref = np.zeros_like(g.F)
    for t, b, d in zip(g.tables, cov.blocks, D):
        O, _ = oracle.conv(t, g.F)
        c, gO = oracle.chi2(oracle.cholesky(b), O, d)
        chi_ref += c
        gF_ref += oracle.conv_grad(t, g.F, gO)
    chi, gF = fit.chi2.cpu().numpy(), fit.gF.cpu().numpy()
    B_chi, B_gF = fit_chain_scales(g.tables, g.F, cov.blocks, D)
    assert np.all(np.abs(chi - chi_ref) <= 1e-12 * B_chi)
    assert np.all(np.abs(gF - gF_ref) <= 1e-12 * B_gF)
    np.testing.assert_allclose(chi, chi_ref, rtol=1e-12)
    assert np.abs(gF - gF_ref).max() <= 1e-12 * np.abs(gF_ref).max()
