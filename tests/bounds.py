"""Componentwise error scales for the FP64 chi^2 chain (test helper).

The contract's "1e-12 relative" is read, for a signed sum, relative to S, the
sum of the absolute values of its terms.  chi^2 and its gradient are not plain
sums but triangular solves (Cholesky factor L of the covariance) applied to a
residual that is itself a difference of nearly equal numbers, so their scale
is the first-order propagation of |terms| through each step (Skeel's
componentwise analysis of substitution: a backward-stable solve of L z = b
satisfies (L + dL) z = b with |dL| <= n u |L|, hence |dz| <= n u |L^-1| |L| |z|):

  residual    r = O - D,                  scale s_r = S_O + |D|
  forward     z = L^-1 r,                 B_z  = |L^-1| (s_r + |L| |z|)
  back        w = L^-T z,                 B_w  = |L^-T| (B_z + |L^T| |w|)
  gradient    gO = 2 w,                   B_g  = 2 B_w
  chi^2       chi2 = z . z,               B_chi = 2 |z| . B_z + z . z
  adjoint     gF = J^T gO,                B_gF = |J|^T (|gO| + B_g)

Two FP64 evaluations that each stay within n u times these scales (n u is at
most ~7e-14 for the block sizes used) differ by far less than 1e-12 of them;
a wrong index, sign or dropped term moves the result by O(1) of them.  The
inverse L^-1 here is numpy's, a library step used for the scale only.
"""
import numpy as np

import oracle
from paper_1909_10547_b300 import workloads as W


def solve_scales(L, res, res_scale=None):
    """L [n][n] lower factor, res [R][n] residuals -> (B_chi [R], B_g [R][n],
    z [R][n], w [R][n]) for chi2 = |L^-1 res|^2 and gO = 2 C^-1 res."""
    L = np.asarray(L, np.float64)
    res = np.atleast_2d(np.asarray(res, np.float64))
    s_r = np.abs(res) if res_scale is None else np.atleast_2d(res_scale)
    Li = np.linalg.inv(L)
    aL, aLi = np.abs(L), np.abs(Li)
    z = res @ Li.T                     # [R][n]
    w = z @ Li                         # L^-T z, row form
    Bz = (s_r + np.abs(z) @ aL.T) @ aLi.T
    Bw = (Bz + np.abs(w) @ aL) @ aLi
    B_chi = 2.0 * (np.abs(z) * Bz).sum(axis=1) + (z * z).sum(axis=1)
    return B_chi, 2.0 * Bw, z, w


def abs_table(t):
    """The table with |FK| (same channels, grid and flavours)."""
    if hasattr(t, "ca"):
        return W.HadTable(np.abs(t.fk), t.ca, t.cb, t.xmap, t.nxg)
    return W.DisTable(np.abs(t.fk), t.flav, t.xmap, t.nxg)


def fit_chain_scales(tables, F, blocks, D_parts):
    """Scales of the fit step's chi^2 [R] and dchi2/dF [R][14][nxg] (one
    covariance block and one D vector per table), from the oracle's forward
    sums S and the propagation above."""
    R = F.shape[0]
    B_chi = np.zeros(R)
    B_gF = np.zeros_like(F)
    aF = np.abs(F)
    for t, b, d in zip(tables, blocks, D_parts):
        O, S = oracle.conv(t, F)
        L = oracle.cholesky(b)
        bc, bg, _, w = solve_scales(L, O - d[None, :], S + np.abs(d)[None, :])
        B_chi += bc
        B_gF += oracle.conv_grad(abs_table(t), aF, np.abs(2.0 * w) + bg)
    return B_chi, B_gF


def ld_solve(L, res):
    """chi^2 and gO = 2 C^-1 res by forward and back substitution in the
    80-bit extended type (numpy longdouble), for checking FP64 results."""
    Lq = np.asarray(L, np.longdouble)
    r = np.atleast_2d(np.asarray(res, np.longdouble))
    R, n = r.shape
    z = np.zeros((R, n), np.longdouble)
    for i in range(n):
        z[:, i] = (r[:, i] - z[:, :i] @ Lq[i, :i]) / Lq[i, i]
    y = np.zeros((R, n), np.longdouble)
    for i in range(n - 1, -1, -1):
        y[:, i] = (z[:, i] - y[:, i + 1:] @ Lq[i + 1:, i]) / Lq[i, i]
    return (z * z).sum(axis=1), 2 * y
