"""Differentiable fit step: autograd wrapper, chi^2 gradient, finite differences.

The fit of the paper is gradient descent (Sec. 2), so the adjoint must give
dchi2/df_a(x_i).  Checks: (1) FKConv.backward equals the oracle gradient;
(2) the fit step's gradient equals the oracle chain (oracle forward, oracle
chi^2 gradient, oracle adjoint); (3) it matches central finite differences of
the GPU chi^2 with h = 1e-6 (absolute, FP64) on sampled coordinates and random
directions, to 1e-6 of max(|g.v|, 1e-3 |g|); (4) the pipelined and the
phase-separated schedules agree with the oracle and replay bit-exactly from
their graphs.
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

SEED = 77


@pytest.fixture(scope="module")
def small_global():
    g = W.config3(R=6, scale=0.12, seed=SEED)
    o_true = [oracle.conv(t, g.F_true)[0][0] for t in g.tables]
    cov = W.covariance(o_true, SEED)
    D = W.pseudo_data(o_true, SEED)
    return g, cov, D


def oracle_chain(g, cov, D, F):
    chi = np.zeros(F.shape[0])
    gF = np.zeros_like(F)
    for t, b, d in zip(g.tables, cov.blocks, D):
        O, _ = oracle.conv(t, F)
        L = oracle.cholesky(b)
        c, gO = oracle.chi2(L, O, d)
        chi += c
        gF += oracle.conv_grad(t, F, gO)
    return chi, gF


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autograd_matches_oracle_gradient(prec):
    t, F = W.config1(R=5, ndata=40, nc=20, nx=16)
    tab = fk.Table.from_workload(t)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Fd = torch.tensor(F, dtype=dt, device="cuda", requires_grad=True)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((5, t.ndata))
    O = fk.FKConv.apply(Fd, tab, prec)
    (O * torch.tensor(w, dtype=dt, device="cuda")).sum().backward()
    ref = oracle.had_grad(t, F, w)
    a = oracle.had_grad(W.HadTable(np.abs(t.fk), t.ca, t.cb, t.xmap, t.nxg), np.abs(F), np.abs(w))
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.all(np.abs(Fd.grad.double().cpu().numpy() - ref) <= tol * a)


@pytest.mark.parametrize("pipelined", [True, False])
def test_fit_step_gradient_matches_oracle_chain(small_global, pipelined):
    """Both schedules: per-table chains on parallel streams, and three phases."""
    g, cov, D = small_global
    fit = GlobalFit(g.tables, g.F, cov.blocks, np.concatenate(D), prec="fp64", pipelined=pipelined)
    fit.step()
    torch.cuda.synchronize()
    chi_ref, gF_ref = oracle_chain(g, cov, D, g.F)
    chi = fit.chi2.cpu().numpy()
    gF = fit.gF.cpu().numpy()
    # 1e-12 of the componentwise scale of the whole chain (forward sums S,
    # residual, both substitutions, adjoint: tests/bounds.py)
    B_chi, B_gF = fit_chain_scales(g.tables, g.F, cov.blocks, D)
    assert np.all(np.abs(chi - chi_ref) <= 1e-12 * B_chi)
    assert np.all(np.abs(gF - gF_ref) <= 1e-12 * B_gF)
    # and plain relative 1e-12: chi^2 per replica, the gradient against its
    # largest entry
    np.testing.assert_allclose(chi, chi_ref, rtol=1e-12)
    assert np.abs(gF - gF_ref).max() <= 1e-12 * np.abs(gF_ref).max()
    print(f"chi2 rel {np.abs(chi / chi_ref - 1).max():.2e}, err/scale {(np.abs(chi - chi_ref) / B_chi).max():.2e}; "
          f"gF rel to max {np.abs(gF - gF_ref).max() / np.abs(gF_ref).max():.2e}, "
          f"err/scale {(np.abs(gF - gF_ref) / np.where(B_gF > 0, B_gF, 1)).max():.2e}")


def test_fit_step_gradient_finite_differences(small_global):
    g, cov, D = small_global
    fit = GlobalFit(g.tables, g.F, cov.blocks, np.concatenate(D), prec="fp64")
    fit.step()
    torch.cuda.synchronize()
    grad = fit.gF.cpu().numpy().copy()
    F0 = fit.F.clone()
    h = 1e-6

    def chi2_at(F):
        fit.F.copy_(torch.tensor(F, device="cuda"))
        fit.step()
        torch.cuda.synchronize()
        return fit.chi2.cpu().numpy().copy()

    rng = np.random.default_rng(3)
    gnorm = np.linalg.norm(grad)
    used = set(int(m) for t in g.tables for m in t.xmap)
    for n in range(24):
        v = np.zeros_like(g.F)
        if n < 16:  # single coordinates on grid points some table uses
            r, a = int(rng.integers(g.F.shape[0])), int(rng.integers(14))
            m = int(rng.choice(sorted(used)))
            v[r, a, m] = 1.0
        else:       # random unit directions
            v = rng.standard_normal(g.F.shape)
            v /= np.linalg.norm(v)
        fd = (chi2_at(g.F + h * v) - chi2_at(g.F - h * v)) / (2 * h)
        gv = (grad * v).sum(axis=(1, 2))
        for r in range(g.F.shape[0]):
            assert abs(fd[r] - gv[r]) <= 1e-6 * max(abs(gv[r]), 1e-3 * gnorm), (n, r, fd[r], gv[r])
    fit.F.copy_(F0)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-3), ("tf32", 5e-2), ("bf16", 0.5)])
def test_fit_step_reduced_precision_chi2(small_global, prec, tol):
    """chi^2 of the reduced-precision fit step against the FP64 oracle; the
    stated error of each mode is a relative bound on chi^2 here."""
    g, cov, D = small_global
    fit = GlobalFit(g.tables, g.F, cov.blocks, np.concatenate(D), prec=prec)
    fit.step()
    torch.cuda.synchronize()
    chi_ref, gF_ref = oracle_chain(g, cov, D, g.F)
    chi = fit.chi2.cpu().numpy()
    rel = np.abs(chi - chi_ref) / np.abs(chi_ref)
    print(prec, "chi2 rel err", rel.max())
    assert rel.max() <= tol


@pytest.mark.parametrize("pipelined", [True, False])
def test_graph_capture_replays_the_step(small_global, pipelined):
    g, cov, D = small_global
    fit = GlobalFit(g.tables, g.F, cov.blocks, np.concatenate(D), prec="fp32", pipelined=pipelined)
    fit.step()
    torch.cuda.synchronize()
    chi_eager = fit.chi2.cpu().numpy().copy()
    gF_eager = fit.gF.cpu().numpy().copy()
    fit.capture()
    fit.chi2.zero_()
    fit.gF.zero_()
    fit.step()
    torch.cuda.synchronize()
    assert np.array_equal(fit.chi2.cpu().numpy(), chi_eager)
    assert np.array_equal(fit.gF.cpu().numpy(), gF_eager)


@pytest.mark.parametrize("prec,tol", [("bf16x3", 2e-4), ("tf32", 2e-2), ("bf16", 0.15)])
def test_fit_step_reduced_precision_gradient(small_global, prec, tol):
    """dchi2/dF of the tensor-core fit step against the FP64 oracle chain,
    relative to the largest gradient entry.  chi^2 weighs the residual O - D,
    a few per cent of O, by C^-1, so an operand rounding of O is amplified in
    the gradient: plain BF16 (measured ~6e-2) is too coarse to fit with, the
    split BF16 operands (~8e-5) are not."""
    g, cov, D = small_global
    fit = GlobalFit(g.tables, g.F, cov.blocks, np.concatenate(D), prec=prec)
    fit.step()
    torch.cuda.synchronize()
    _, gF_ref = oracle_chain(g, cov, D, g.F)
    err = np.abs(fit.gF.double().cpu().numpy() - gF_ref).max() / np.abs(gF_ref).max()
    print(prec, "gradient rel err", err)
    assert err <= tol


@pytest.mark.parametrize("pipelined", [True, False])
def test_saved_products_do_not_change_the_step(small_global, pipelined):
    """The step with the forward's saved products (the default in the
    tensor-core modes) gives the chi^2 and gradient of the step without
    them, bit for bit, eager and replayed from its graph."""
    g, cov, D = small_global
    res = []
    for save in (False, True):
        fit = GlobalFit(g.tables, g.F, cov.blocks, np.concatenate(D), prec="bf16x3", pipelined=pipelined,
                        save_products=save)
        assert any(b is not None for b in fit.saved) == save
        fit.step()
        torch.cuda.synchronize()
        res.append((fit.chi2.cpu().numpy().copy(), fit.gF.cpu().numpy().copy()))
        if save:
            fit.capture()
            fit.chi2.zero_()
            fit.gF.zero_()
            fit.step()
            torch.cuda.synchronize()
            res.append((fit.chi2.cpu().numpy().copy(), fit.gF.cpu().numpy().copy()))
    for chi, gF in res[1:]:
        assert np.array_equal(chi, res[0][0])
        assert np.array_equal(gF, res[0][1])


def test_whitened_tables(small_global):
    """whiten_tables (the dense FP64 product on the device) gives L^{-1} FK and
    L^{-1} D of each dataset as forward substitution with the same factor L
    does (a componentwise-accurate solve: a pivoting LU solve is not, its row 0
    picks up the rounding of the larger rows).  Both carry errors of order
    kappa(L) u64 of the componentwise scale |L^{-1}| |FK|; they agree to 1e-10
    of it, where a wrong index or transpose would be off by O(1).  (Another
    factorisation of C differs from L by kappa(C) u64, which L^{-1} can amplify
    past that bound, so the reference uses numpy's, as whiten_tables does.)"""
    from scipy.linalg import solve_triangular

    from paper_1909_10547_b300.fitstep import whiten_tables
    g, cov, D = small_global
    wt, Dw = whiten_tables(g.tables, cov.blocks, D)
    for t, w, b, d, dw in zip(g.tables, wt, cov.blocks, D, Dw):
        L = np.linalg.cholesky(b)
        n = t.ndata
        ref = solve_triangular(L, t.fk.reshape(n, -1), lower=True).reshape(t.fk.shape)
        aLi = np.abs(solve_triangular(L, np.eye(n), lower=True))
        scale = aLi @ np.abs(t.fk.reshape(n, -1))
        assert np.all(np.abs(w.fk - ref).reshape(n, -1) <= 1e-10 * scale)
        assert np.all(np.abs(dw - solve_triangular(L, d, lower=True)) <= 1e-10 * (aLi @ np.abs(d)))
        assert type(w) is type(t) and w.fk.shape == t.fk.shape


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-4)])
def test_whitened_step_matches_plain(small_global, prec, tol):
    """The step on whitened tables (the default in the non-FP64 modes) gives
    the chi^2 and gradient of the step with the substitutions: the same
    quantities, rounded differently (relative to the oracle's scales)."""
    g, cov, D = small_global
    res = []
    for whiten in (False, True):
        fit = GlobalFit(g.tables, g.F, cov.blocks, np.concatenate(D), prec=prec, whiten=whiten)
        assert fit.whiten == whiten
        fit.step()
        torch.cuda.synchronize()
        res.append((fit.chi2.cpu().numpy().copy(), fit.gF.double().cpu().numpy().copy()))
    chi_ref, gF_ref = oracle_chain(g, cov, D, g.F)
    (c0, g0), (c1, g1) = res
    for c, gg in res:
        assert np.abs(c - chi_ref).max() <= tol * np.abs(chi_ref).max()
        assert np.abs(gg - gF_ref).max() <= 2 * tol * np.abs(gF_ref).max()
    print(prec, "chi2 rel err plain", (np.abs(c0 - chi_ref) / np.abs(chi_ref)).max(),
          "whitened", (np.abs(c1 - chi_ref) / np.abs(chi_ref)).max(),
          "grad rel err plain", np.abs(g0 - gF_ref).max() / np.abs(gF_ref).max(),
          "whitened", np.abs(g1 - gF_ref).max() / np.abs(gF_ref).max())
