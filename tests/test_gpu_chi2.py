"""FP64 chi^2 on the device vs the oracle (Cholesky-Banachiewicz + substitution).

Tolerance: 1e-12 of the componentwise scale of each result (tests/bounds.py:
the propagation of |terms| through the forward and back substitutions), the
reading of "1e-12 relative" for a triangular solve; chi^2 also meets plain
relative 1e-12 on these blocks."""
import numpy as np
import pytest
import torch

import oracle
import paper_1909_10547_b300 as fk
from paper_1909_10547_b300 import workloads as W

from bounds import solve_scales

pytestmark = pytest.mark.gpu


def _blocks(sizes, seed):
    rng = np.random.default_rng(seed)
    o = [rng.uniform(0.5, 5.0, n) for n in sizes]
    return W.covariance(o, seed), o


@pytest.mark.parametrize("sizes,R", [([1], 1), ([2, 3], 2), ([31, 33, 64, 65], 33),
                                     ([600, 10, 250], 100), ([17] * 40, 7)])
def test_chi2_matches_oracle(sizes, R):
    cov, o = _blocks(sizes, len(sizes) + R)
    D = np.concatenate(W.pseudo_data(o, 5))
    rng = np.random.default_rng(R)
    O = np.concatenate(o)[None, :] * rng.uniform(0.9, 1.1, (R, sum(sizes)))
    want = np.zeros(R)
    B_chi = np.zeros(R)
    g_want = np.zeros((R, sum(sizes)))
    B_g = np.zeros((R, sum(sizes)))
    off = 0
    for b in cov.blocks:
        n = b.shape[0]
        L = oracle.cholesky(b)
        c, g = oracle.chi2(L, O[:, off:off + n], D[off:off + n])
        want += c
        g_want[:, off:off + n] = g
        bc, bg, _, _ = solve_scales(L, O[:, off:off + n] - D[None, off:off + n])
        B_chi += bc
        B_g[:, off:off + n] = bg
        off += n
    dc = fk.Cov(cov.blocks)
    Od = torch.tensor(O, device="cuda")
    Dd = torch.tensor(D, device="cuda")
    c, g = fk.chi2(dc, Od, Dd)
    torch.cuda.synchronize()
    c, g = c.cpu().numpy(), g.cpu().numpy()
    np.testing.assert_allclose(c, want, rtol=1e-12, atol=0)
    assert np.all(np.abs(c - want) <= 1e-12 * B_chi)
    assert np.all(np.abs(g - g_want) <= 1e-12 * B_g)
    # and plain relative 1e-12 of each replica's largest gradient entry
    assert np.all(np.abs(g - g_want) <= 1e-12 * np.abs(g_want).max(axis=1, keepdims=True))
    rel = np.abs(g - g_want).max() / np.abs(g_want).max()
    print(f"sizes {sizes}: chi2 rel {np.abs(c / want - 1).max():.2e}, gO rel to max {rel:.2e}, "
          f"gO err / scale {(np.abs(g - g_want) / B_g).max():.2e}")


@pytest.mark.parametrize("R", [1, 9, 300])
def test_chi2_result_independent_of_R(R):
    """A replica's chi^2 and gradient do not depend on which replicas share
    the call (the solve's sums run in an order fixed by the block alone)."""
    sizes = [150, 40]
    cov, o = _blocks(sizes, 4)
    D = np.concatenate(W.pseudo_data(o, 4))
    rng = np.random.default_rng(8)
    O = np.concatenate(o)[None, :] * rng.uniform(0.9, 1.1, (R, sum(sizes)))
    dc = fk.Cov(cov.blocks)
    Dd = torch.tensor(D, device="cuda")
    c, g = fk.chi2(dc, torch.tensor(O, device="cuda"), Dd)
    c1, g1 = fk.chi2(dc, torch.tensor(O[-1:], device="cuda"), Dd)
    assert c[-1].item() == c1[0].item()
    assert torch.equal(g[-1], g1[0])


def test_chi2_zero_at_data_and_identity_cov():
    n = 50
    D = np.linspace(1, 2, n)
    dc = fk.Cov([np.eye(n)])
    O = np.stack([D, D + 1.0, D * 2])
    c, g = fk.chi2(dc, torch.tensor(O, device="cuda"), torch.tensor(D, device="cuda"))
    c, g = c.cpu().numpy(), g.cpu().numpy()
    assert c[0] == 0.0 and np.all(g[0] == 0.0)
    assert abs(c[1] - n) < 1e-12 * n
    np.testing.assert_allclose(c[2], ((D) ** 2).sum(), rtol=1e-13)
    np.testing.assert_allclose(g[2], 2 * D, rtol=1e-14)


@pytest.mark.parametrize("sizes,R", [([600, 10, 250], 100), ([31, 33, 64, 65], 33), ([1], 1), ([2100, 5], 3)])
def test_chi2_fp32_io_matches_oracle(sizes, R):
    """FP32 observables and gradient (the reduced-mode fit).  The arithmetic is
    FP64 as for FP64 outputs, so against the oracle on the same FP32-rounded O
    chi^2 (FP64 out) meets the 1e-12 contract of its componentwise scale and
    gO is within its FP32 rounding plus that."""
    cov, o = _blocks(sizes, len(sizes) + R + 11)
    D = np.concatenate(W.pseudo_data(o, 6))
    rng = np.random.default_rng(R + 5)
    O32 = (np.concatenate(o)[None, :] * rng.uniform(0.9, 1.1, (R, sum(sizes)))).astype(np.float32)
    O = O32.astype(np.float64)
    want, B_chi = np.zeros(R), np.zeros(R)
    g_want, B_g = np.zeros((R, sum(sizes))), np.zeros((R, sum(sizes)))
    off = 0
    for b in cov.blocks:
        n = b.shape[0]
        L = oracle.cholesky(b)
        c, g = oracle.chi2(L, O[:, off:off + n], D[off:off + n])
        want += c
        g_want[:, off:off + n] = g
        bc, bg, _, _ = solve_scales(L, O[:, off:off + n] - D[None, off:off + n])
        B_chi += bc
        B_g[:, off:off + n] = bg
        off += n
    dc = fk.Cov(cov.blocks)
    c, g = fk.chi2(dc, torch.tensor(O32, device="cuda"), torch.tensor(D, device="cuda"))
    torch.cuda.synchronize()
    assert g.dtype == torch.float32
    c, g = c.cpu().numpy(), g.double().cpu().numpy()
    assert np.all(np.abs(c - want) <= 1e-12 * B_chi), (np.abs(c - want) / B_chi).max()
    assert np.all(np.abs(g - g_want) <= 2.0 ** -24 * np.abs(g_want) + 1e-12 * B_g)
    print(f"sizes {sizes}: chi2 err / scale {(np.abs(c - want) / B_chi).max():.2e}, "
          f"gO err / |gO| {(np.abs(g - g_want) / np.maximum(np.abs(g_want), 1e-300)).max():.2e}")


def test_chi2_fp32_io_independent_of_R():
    sizes = [150, 40]
    cov, o = _blocks(sizes, 9)
    D = torch.tensor(np.concatenate(W.pseudo_data(o, 9)), device="cuda")
    O = np.concatenate(o)[None, :] * np.random.default_rng(2).uniform(0.9, 1.1, (300, sum(sizes)))
    Od = torch.tensor(O, dtype=torch.float32, device="cuda")
    dc = fk.Cov(cov.blocks)
    c, g = fk.chi2(dc, Od, D)
    c1, g1 = fk.chi2(dc, Od[-1:].contiguous(), D)
    assert c[-1].item() == c1[0].item()
    assert torch.equal(g[-1], g1[0])


@pytest.mark.parametrize("sizes,R,dtype", [([600, 10, 250], 100, torch.float64), ([31, 33], 7, torch.float32),
                                           ([1], 1, torch.float64)])
def test_chi2_white_matches_oracle(sizes, R, dtype):
    """chi^2 of whitened observables: with Z = L^{-1} O and Dw = L^{-1} D
    (formed here in FP64 on the host), |Z - Dw|^2 is the oracle's
    (O - D)^T C^{-1} (O - D) within 1e-12 of its scale, and d chi2/dZ = 2 z is
    L^T times the oracle's d chi2/dO (2 L^-T z)."""
    cov, o = _blocks(sizes, len(sizes) + R + 3)
    D = np.concatenate(W.pseudo_data(o, 7))
    rng = np.random.default_rng(R + 9)
    O = np.concatenate(o)[None, :] * rng.uniform(0.9, 1.1, (R, sum(sizes)))
    if dtype == torch.float32:
        O = O.astype(np.float32).astype(np.float64)
    Z, Dw, want, B_chi = np.zeros_like(O), np.zeros_like(D), np.zeros(R), np.zeros(R)
    gz_want = np.zeros_like(O)
    off = 0
    for b in cov.blocks:
        n = b.shape[0]
        L = oracle.cholesky(b)
        c, g = oracle.chi2(L, O[:, off:off + n], D[off:off + n])
        want += c
        Z[:, off:off + n] = np.linalg.solve(L, O[:, off:off + n].T).T
        Dw[off:off + n] = np.linalg.solve(L, D[off:off + n])
        gz_want[:, off:off + n] = g @ L  # dchi2/dZ = L^T dchi2/dO, row form
        bc, _, _, _ = solve_scales(L, O[:, off:off + n] - D[None, off:off + n])
        B_chi += bc
        off += n
    Zd = torch.tensor(Z, dtype=dtype, device="cuda")
    c, gz = fk.chi2_white(Zd, torch.tensor(Dw, device="cuda"))
    torch.cuda.synchronize()
    c, gz = c.cpu().numpy(), gz.double().cpu().numpy()
    if dtype == torch.float32:  # Z itself rounded to FP32: compare with its own exact sum
        Zr = Zd.double().cpu().numpy()
        want = ((Zr - Dw) ** 2).sum(axis=1)
        np.testing.assert_allclose(c, want, rtol=1e-13)
        np.testing.assert_allclose(gz, (2 * (Zr - Dw)).astype(np.float32), rtol=0, atol=0)
        return
    assert np.all(np.abs(c - want) <= 1e-12 * B_chi), (np.abs(c - want) / B_chi).max()
    assert np.abs(gz - gz_want).max() <= 1e-12 * np.abs(gz_want).max()


def test_chi2_white_strides_and_errors():
    Z = torch.tensor(np.random.default_rng(3).standard_normal((5, 12)), device="cuda")
    Dw = torch.tensor(np.random.default_rng(4).standard_normal(7), device="cuda")
    c, g = fk.chi2_white(Z[:, 2:9], Dw)
    ref = ((Z[:, 2:9].cpu().numpy() - Dw.cpu().numpy()) ** 2).sum(axis=1)
    np.testing.assert_allclose(c.cpu().numpy(), ref, rtol=1e-14)
    assert torch.equal(g, 2 * (Z[:, 2:9] - Dw))
    with pytest.raises(ValueError):
        fk.chi2_white(Z, Dw)  # Dw of the wrong length


def test_cov_rejects_non_spd():
    bad = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(fk.FKError, match="positive definite"):
        fk.Cov([np.eye(3), bad])
