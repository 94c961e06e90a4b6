"""Gradient-descent fit of parametrised PDFs over the global set.

The paper fits PDFs by gradient descent on chi^2 (Sec. 2).  Here each replica
r has its own parameters theta[r][a] = (ln A, alpha, beta) per flavour a, with
f^r_a(x) = A x^alpha (1 - x)^beta on the master x grid (the analytic form
stands in for the paper's neural network).  One iteration:

  fk_pdf_eval    theta -> F                      (library kernel)
  GlobalFit      F -> chi2, dchi2/dF             (forward, FP64 chi^2, adjoint)
  fk_pdf_grad    dchi2/dF -> dchi2/dtheta        (library kernel)
  fk_adam_step   theta -= Adam(dchi2/dtheta)     (library kernel)

The replicas are independent fits running side by side in every launch.
"""
import ctypes

import numpy as np
import torch

from . import _lib, _p, _prec, _stream
from .fitstep import GlobalFit

NFL = 14


def pdf_eval(theta, x_grid, F, prec):
    """F[r][a][m] = exp(t0 + t1 ln x_m + t2 ln(1 - x_m)) (fk_pdf_eval)."""
    _lib.call("fk_pdf_eval", _p(theta), theta.shape[0], _p(x_grid), x_grid.numel(), _p(F), _prec(prec),
              _stream())
    return F


def pdf_grad(F, gF, x_grid, gtheta, prec):
    """dchi2/dtheta from dchi2/dF through the parametrisation (fk_pdf_grad)."""
    _lib.call("fk_pdf_grad", _p(F), _p(gF), F.shape[0], _p(x_grid), x_grid.numel(), _p(gtheta), _prec(prec),
              _stream())
    return gtheta


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, prec="fp32"):
    """One Adam step in place (fk_adam_step)."""
    _lib.call("fk_adam_step", _p(p), _p(g), _p(m), _p(v), ctypes.c_longlong(p.numel()), int(t),
              ctypes.c_double(lr), ctypes.c_double(b1), ctypes.c_double(b2), ctypes.c_double(eps), _prec(prec),
              _stream())


class PDFDescent:
    """Adam on the PDF parameters of every replica, with the fit step of
    `fit` (a GlobalFit whose F buffer the parametrisation writes)."""

    def __init__(self, fit: GlobalFit, theta0: np.ndarray, x_grid: np.ndarray, lr=0.02,
                 b1=0.9, b2=0.999, eps=1e-8):
        self.fit = fit
        dev = fit.F.device
        self.prec = fit.prec
        self.theta = torch.tensor(np.asarray(theta0), dtype=fit.io, device=dev).contiguous()
        assert self.theta.shape == (fit.R, NFL, 3)
        self.x = torch.tensor(np.asarray(x_grid, np.float64), device=dev)
        assert self.x.numel() == fit.nxg
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.g = torch.empty_like(self.theta)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self):
        """One iteration; afterwards fit.chi2 holds chi^2 at the parameters
        the iteration started from."""
        pdf_eval(self.theta, self.x, self.fit.F, self.prec)
        self.fit.step()
        pdf_grad(self.fit.F, self.fit.gF, self.x, self.g, self.prec)
        self.t += 1
        adam_step(self.theta, self.g, self.m, self.v, self.t, self.lr, self.b1, self.b2, self.eps, self.prec)

    def run(self, iters, every=10):
        """Runs `iters` iterations; returns the chi^2 of every replica at
        iterations 0, every, 2 every, ... as an array [k][R]."""
        hist = []
        for k in range(iters):
            self.step()
            if k % every == 0 or k == iters - 1:
                hist.append(self.fit.chi2.double().cpu().numpy().copy())
        return np.array(hist)
