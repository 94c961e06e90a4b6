"""Host side of the whitened fit step (no GPU).

With C = L L^T, chi2 = (O - D)^T C^{-1} (O - D) = |L^{-1} O - L^{-1} D|^2 and
d chi2 / dO = L^{-T} d chi2 / dZ for Z = L^{-1} O: the identity the fit step
on whitened tables rests on.  Checked against the oracle's substitution
chi^2 (its own Cholesky and solves), together with the lower-triangular
inverse that whiten_tables forms on the host.
"""
import numpy as np
import pytest
from scipy.linalg import solve_triangular

import oracle
from paper_1909_10547_b300 import workloads as W
from paper_1909_10547_b300.fitstep import _lower_inverse

from bounds import solve_scales


@pytest.mark.parametrize("n", [1, 2, 7, 33, 150])
def test_lower_inverse(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    L = np.linalg.cholesky(A @ A.T + n * np.eye(n))
    X = _lower_inverse(L)
    assert np.all(np.triu(X, 1) == 0.0)  # exact zeros above the diagonal
    ref = solve_triangular(L, np.eye(n), lower=True)
    scale = np.abs(ref) @ np.abs(L) @ np.abs(ref)  # componentwise scale of an inverse
    assert np.all(np.abs(X - ref) <= 1e-13 * scale)
    np.testing.assert_allclose(X @ L, np.eye(n), atol=1e-12)


@pytest.mark.parametrize("n,R", [(1, 1), (12, 3), (90, 5)])
def test_whitened_chi2_is_the_oracle_chi2(n, R):
    o = np.random.default_rng(n + R).uniform(0.5, 5.0, n)
    cov = W.covariance([o], n)
    C = cov.blocks[0]
    D = W.pseudo_data([o], n)[0]
    O = o[None, :] * np.random.default_rng(R).uniform(0.9, 1.1, (R, n))
    L = oracle.cholesky(C)
    chi_ref, g_ref = oracle.chi2(L, O, D)
    Li = _lower_inverse(np.linalg.cholesky(C))
    z = O @ Li.T - Li @ D          # Z - Dw, row form
    chi = (z * z).sum(axis=1)
    g = (2.0 * z) @ Li             # L^{-T} (2 z), row form: d chi2 / dO
    B_chi, B_g, _, _ = solve_scales(L, O - D[None, :])
    assert np.all(np.abs(chi - chi_ref) <= 1e-12 * B_chi)
    assert np.all(np.abs(g - g_ref) <= 1e-12 * B_g)
