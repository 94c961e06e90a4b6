"""Gradient descent over PDF parameters (fk_pdf_eval, fk_pdf_grad,
fk_adam_step and the loop in descent.py).

The fit of the paper minimises chi^2 by gradient descent (Sec. 2).  Checks:
the parametrisation and its adjoint against their definition and against
central finite differences; the Adam step against a plain restatement of the
published update; and an end-to-end descent on a scaled global set that must
lower every replica's chi^2 by a large factor, in FP64 and in BF16 hi+lo.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1909_10547_b300 import workloads as W
from paper_1909_10547_b300.descent import PDFDescent, adam_step, pdf_eval, pdf_grad
from paper_1909_10547_b300.fitstep import GlobalFit

pytestmark = pytest.mark.gpu

X = W.xgrid(50, 1e-7)


def _theta(rng, R):
    t = np.empty((R, 14, 3))
    t[..., 0] = rng.uniform(-0.7, 0.7, (R, 14))
    t[..., 1] = rng.uniform(-0.2, 0.8, (R, 14))
    t[..., 2] = rng.uniform(1.0, 5.0, (R, 14))
    return t


def _F_ref(t):
    return np.exp(t[..., 0:1] + t[..., 1:2] * np.log(X) + t[..., 2:3] * np.log1p(-X))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_pdf_eval_and_grad_match_definition(prec, tol):
    rng = np.random.default_rng(3)
    dt = torch.float64 if prec == "fp64" else torch.float32
    t = _theta(rng, 4)
    th = torch.tensor(t, dtype=dt, device="cuda")
    x = torch.tensor(X, device="cuda")
    F = torch.empty((4, 14, 50), dtype=dt, device="cuda")
    pdf_eval(th, x, F, prec)
    Fr = _F_ref(t)
    assert np.all(np.abs(F.double().cpu().numpy() - Fr) <= tol * np.abs(Fr))
    gF = rng.standard_normal((4, 14, 50))
    g = torch.empty_like(th)
    pdf_grad(F, torch.tensor(gF, dtype=dt, device="cuda"), x, g, prec)
    w = gF * Fr
    ref = np.stack([w.sum(-1), (w * np.log(X)).sum(-1), (w * np.log1p(-X)).sum(-1)], -1)
    scale = np.stack([np.abs(w).sum(-1), (np.abs(w) * np.abs(np.log(X))).sum(-1),
                      (np.abs(w) * np.abs(np.log1p(-X))).sum(-1)], -1)
    assert np.all(np.abs(g.double().cpu().numpy() - ref) <= 10 * tol * scale)


def test_pdf_grad_finite_differences():
    """d/dtheta of L(theta) = sum gF * F(theta) by central differences (FP64)."""
    rng = np.random.default_rng(5)
    t = _theta(rng, 2)
    gF = rng.standard_normal((2, 14, 50))
    x = torch.tensor(X, device="cuda")
    F = torch.empty((2, 14, 50), dtype=torch.float64, device="cuda")
    pdf_eval(torch.tensor(t, device="cuda"), x, F, "fp64")
    g = torch.empty((2, 14, 3), dtype=torch.float64, device="cuda")
    pdf_grad(F, torch.tensor(gF, device="cuda"), x, g, "fp64")
    g = g.cpu().numpy()

    def L(tt):
        Fd = torch.empty((2, 14, 50), dtype=torch.float64, device="cuda")
        pdf_eval(torch.tensor(tt, device="cuda"), x, Fd, "fp64")
        return float((Fd.cpu().numpy() * gF).sum())

    h = 1e-6
    for (r, a, k) in [(0, 0, 0), (0, 3, 1), (1, 7, 2), (1, 13, 1), (0, 9, 2)]:
        tp, tm = t.copy(), t.copy()
        tp[r, a, k] += h
        tm[r, a, k] -= h
        fd = (L(tp) - L(tm)) / (2 * h)
        assert abs(fd - g[r, a, k]) <= 1e-6 * max(abs(g[r, a, k]), 1.0), (r, a, k, fd, g[r, a, k])


def test_adam_matches_the_published_update():
    rng = np.random.default_rng(7)
    n = 1000
    p = rng.standard_normal(n)
    m = np.zeros(n)
    v = np.zeros(n)
    pd, md, vd = (torch.tensor(a, device="cuda") for a in (p, m, v))
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    for t in range(1, 6):
        g = rng.standard_normal(n)
        adam_step(pd, torch.tensor(g, device="cuda"), md, vd, t, lr, b1, b2, eps, prec="fp64")
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    np.testing.assert_allclose(pd.cpu().numpy(), p, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(md.cpu().numpy(), m, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(vd.cpu().numpy(), v, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_descent_lowers_chi2(prec):
    """Replicas start from jittered parameters; Adam on the PDF parameters
    must lower every replica's chi^2 by a large factor."""
    R = 6
    g = W.config3(R=R, scale=0.12, seed=31)
    o_true = [oracle.conv(t, g.F_true)[0][0] for t in g.tables]
    cov = W.covariance(o_true, 31)
    D = np.concatenate(W.pseudo_data(o_true, 31))
    rng = np.random.default_rng(11)
    t0 = np.empty((R, 14, 3))
    t0[..., 0] = np.log(g.params.A)[None, :] + rng.uniform(-0.3, 0.3, (R, 14))
    t0[..., 1] = g.params.alpha[None, :] * rng.uniform(0.8, 1.2, (R, 14))
    t0[..., 2] = g.params.beta[None, :] * rng.uniform(0.8, 1.2, (R, 14))
    fit = GlobalFit(g.tables, np.zeros((R, 14, 50)), cov.blocks, D, prec=prec)
    gd = PDFDescent(fit, t0, g.x, lr=0.02)
    hist = gd.run(300, every=50)
    first, last = hist[0], hist[-1]
    print(prec, "chi2 first", first, "last", last)
    assert np.all(np.isfinite(last))
    assert np.all(last < first / 20)
