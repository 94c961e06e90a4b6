"""The componentwise scales of tests/bounds.py, checked on the CPU.

(1) The oracle's FP64 chi^2 and gradient lie within 1e-13 of those scales of
an independent forward/back substitution in the 80-bit extended type, so the
1e-12 tolerance the GPU tests apply with them leaves the oracle's own error
far inside.  (2) The scales are not vacuous: plausible mistakes in a solve
(a dropped entry of L, the factor 2 of the gradient, a transposed factor, a
shifted residual) move the result by many orders more than 1e-12 of them.
"""
import numpy as np
import pytest

import oracle
from paper_1909_10547_b300 import workloads as W

from bounds import ld_solve, solve_scales


def _case(n, R, seed):
    rng = np.random.default_rng(seed)
    o = [rng.uniform(0.5, 5.0, n)]
    C = W.covariance(o, seed).blocks[0]
    D = W.pseudo_data(o, seed)[0]
    O = o[0][None, :] * rng.uniform(0.9, 1.1, (R, n))
    return C, D, O


@pytest.mark.parametrize("n,R", [(1, 2), (7, 3), (33, 4), (200, 3)])
def test_oracle_within_scale_of_extended_precision(n, R):
    C, D, O = _case(n, R, n)
    L = oracle.cholesky(C)
    c, g = oracle.chi2(L, O, D)
    c_ld, g_ld = ld_solve(L, O - D[None, :])
    B_chi, B_g, _, _ = solve_scales(L, O - D[None, :])
    assert np.all(np.abs(c - c_ld.astype(np.float64)) <= 1e-13 * B_chi)
    assert np.all(np.abs(g - g_ld.astype(np.float64)) <= 1e-13 * B_g)


def test_scales_detect_planted_mistakes():
    n, R = 60, 3
    C, D, O = _case(n, R, 11)
    L = oracle.cholesky(C)
    res = O - D[None, :]
    c, g = oracle.chi2(L, O, D)
    B_chi, B_g, _, _ = solve_scales(L, res)

    def far(c2, g2):
        return (np.abs(c2 - c) / B_chi).max() > 1e-6 or (np.abs(g2 - g) / B_g).max() > 1e-6

    L1 = L.copy()
    L1[40, 17] = 0.0                       # a dropped term of the substitution
    assert far(*oracle.chi2(L1, O, D))
    assert far(c, g / 2)                   # the gradient's factor 2
    L2 = np.tril(L.T)                      # factor read from the wrong triangle: only the diagonal left
    assert far(*oracle.chi2(L2, O, D))
    Dm = np.roll(D, 1)                     # residual against a shifted data vector
    assert far(*oracle.chi2(L, O, Dm))


def test_scale_of_identity_covariance_is_the_plain_sum():
    """With C = I the solve is the identity: B_chi = 5 sum r^2 (the residual's
    rounding, its propagation and the sum), B_g = 2 (2 |r| + |r|) per entry."""
    r = np.array([[1.0, -2.0, 0.5]])
    B_chi, B_g, z, w = solve_scales(np.eye(3), r)
    assert np.allclose(z, r) and np.allclose(w, r)
    assert np.isclose(B_chi[0], 2 * (np.abs(r) * 2 * np.abs(r)).sum() + (r * r).sum())
    assert np.allclose(B_g, 2 * (2 * np.abs(r) + np.abs(r)))
