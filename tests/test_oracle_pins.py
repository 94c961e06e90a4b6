"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each uses an independent route
(hand-worked values, exact rational brute force, closed forms, invariants of a
linear or quadratic form, a library special case) chosen so that a dropped
term, a swapped index or a transposed operand in the oracle fails a test.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1909_10547_b300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")


class T:
    """Minimal table record accepted by the oracle wrappers."""

    def __init__(self, fk, xmap=None, nxg=None, ca=None, cb=None):
        self.fk = np.asarray(fk, np.float64)
        nx = self.fk.shape[-1]
        self.xmap = np.arange(nx, dtype=np.int32) if xmap is None else np.asarray(xmap, np.int32)
        self.nxg = nx if nxg is None else nxg
        if ca is not None:
            self.ca = np.asarray(ca, np.int32)
            self.cb = np.asarray(cb, np.int32)


# ---------------------------------------------------------------- golden ----

def test_golden_hadronic_hand_worked():
    g = json.load(open(GOLD))["hadronic"]
    ca = [c[0] for c in g["channels"]]
    cb = [c[1] for c in g["channels"]]
    t = T(g["fk"], ca=ca, cb=cb)
    F = np.zeros((1, 14, g["nx"]))
    for a, v in g["pdf"].items():
        F[0, int(a)] = v
    O, _ = oracle.had(t, F)
    assert O[0].tolist() == g["O"]
    gF = oracle.had_grad(t, F, np.ones((1, 1)))
    for a in range(14):
        want = g["grad"].get(str(a), [0, 0])
        assert gF[0, a].tolist() == want, a


def test_golden_dis_hand_worked():
    g = json.load(open(GOLD))["dis"]
    fk = np.zeros((g["ndata"], 14, g["nx"]))
    for d, row in g["fk_nonzero"].items():
        for a, v in row.items():
            fk[int(d), int(a)] = v
    F = np.zeros((1, 14, g["nx"]))
    for a, v in g["pdf"].items():
        F[0, int(a)] = v
    t = T(fk)
    O, _ = oracle.dis(t, F)
    assert O[0].tolist() == g["O"]
    gF = oracle.dis_grad(t, np.array([g["gO"]], np.float64))
    for a in range(14):
        assert gF[0, a].tolist() == g["grad"].get(str(a), [0, 0]), a


def test_golden_chi2_hand_worked():
    g = json.load(open(GOLD))["chi2"]
    L = oracle.cholesky(np.array(g["C"], np.float64))
    np.testing.assert_allclose(L, np.array(g["L"]), rtol=0, atol=1e-15)
    r = np.array([g["O_minus_D"]], np.float64)
    c, gO = oracle.chi2(L, r, np.zeros(2))
    assert abs(c[0] - g["chi2"]) < 1e-15
    np.testing.assert_allclose(gO[0], g["gO"], rtol=0, atol=1e-15)


# ---------------------------------------------------- exact brute force ----

def _frac_had(fk, ca, cb, xmap, F):
    """Exact rational value of Eq. 1, written as one sum over (c, i, j)."""
    nd, nc, nx, _ = fk.shape
    R = F.shape[0]
    out = [[Fraction(0)] * nd for _ in range(R)]
    for r in range(R):
        for d in range(nd):
            s = Fraction(0)
            for c in range(nc):
                for i in range(nx):
                    for j in range(nx):
                        s += (Fraction(int(fk[d, c, i, j])) * Fraction(int(F[r, ca[c], xmap[i]]))
                              * Fraction(int(F[r, cb[c], xmap[j]])))
            out[r][d] = s
    return out


def _tiny_int_had(seed, nd=3, nc=4, nx=3, nxg=5, R=3, lo=-4, hi=5):
    rng = np.random.default_rng(seed)
    pairs = rng.choice(196, nc, replace=False)
    ca, cb = (pairs // 14).astype(np.int32), (pairs % 14).astype(np.int32)
    # force one diagonal channel so the product rule on a == b is exercised
    ca[0] = cb[0]
    if len(set(zip(ca.tolist(), cb.tolist()))) < nc:
        ca[0], cb[0] = 13, 13
    fk = rng.integers(lo, hi, (nd, nc, nx, nx)).astype(np.float64)
    xmap = np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32)
    F = rng.integers(lo, hi, (R, 14, nxg)).astype(np.float64)
    return T(fk, xmap, nxg, ca, cb), F


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_had_exact_bruteforce(seed):
    t, F = _tiny_int_had(seed)
    O, S = oracle.had(t, F)
    ref = _frac_had(t.fk, t.ca, t.cb, t.xmap, F)
    assert O.tolist() == [[float(v) for v in row] for row in ref]
    assert np.all(S >= np.abs(O))


@pytest.mark.parametrize("seed", [4, 5])
def test_had_grad_exact_central_difference(seed):
    """Eq. 1 is quadratic in f, so a central difference with step 1 is its
    exact derivative; evaluated with rationals it pins the gradient."""
    t, F = _tiny_int_had(seed, R=2)
    rng = np.random.default_rng(seed + 100)
    gO = rng.integers(-3, 4, (2, t.fk.shape[0])).astype(np.float64)
    gF = oracle.had_grad(t, F, gO)
    for r in range(2):
        for a in range(14):
            for m in range(t.nxg):
                Fp = F.copy()
                Fm = F.copy()
                Fp[r, a, m] += 1
                Fm[r, a, m] -= 1
                op = _frac_had(t.fk, t.ca, t.cb, t.xmap, Fp[r:r + 1])[0]
                om = _frac_had(t.fk, t.ca, t.cb, t.xmap, Fm[r:r + 1])[0]
                want = sum(Fraction(int(gO[r, d])) * (op[d] - om[d]) / 2 for d in range(len(op)))
                assert gF[r, a, m] == float(want), (r, a, m)


def test_dis_exact_bruteforce_and_grad():
    rng = np.random.default_rng(7)
    nd, nx, nxg, R = 4, 3, 6, 3
    fk = rng.integers(-5, 6, (nd, 14, nx)).astype(np.float64)
    fk[:, [2, 9], :] = 0.0  # inactive flavours
    xmap = np.array([0, 2, 5], np.int32)
    F = rng.integers(-5, 6, (R, 14, nxg)).astype(np.float64)
    t = T(fk, xmap, nxg)
    O, _ = oracle.dis(t, F)
    for r in range(R):
        for d in range(nd):
            want = sum(Fraction(int(fk[d, a, i])) * Fraction(int(F[r, a, xmap[i]]))
                       for a in range(14) for i in range(nx))
            assert O[r, d] == float(want)
    gO = rng.integers(-3, 4, (R, nd)).astype(np.float64)
    gF = oracle.dis_grad(t, gO)
    for r in range(R):
        for a in range(14):
            for m in range(nxg):
                want = 0
                if m in xmap.tolist():
                    i = xmap.tolist().index(m)
                    want = sum(int(gO[r, d]) * int(fk[d, a, i]) for d in range(nd))
                assert gF[r, a, m] == want


# ------------------------------------------------------------ delta PDFs ----

def _had_float(seed=11, nd=5, nc=7, nx=6):
    rng = np.random.default_rng(seed)
    x = W.xgrid(nx, 1e-6)
    return W.had_table(rng, nd, nc, x)


def test_had_delta_pdf_returns_diagonal_slice():
    t = _had_float()
    pairs = list(zip(t.ca.tolist(), t.cb.tolist()))
    t.ca[0] = t.cb[0] = 5  # make sure one diagonal channel exists
    pairs = list(zip(t.ca.tolist(), t.cb.tolist()))
    for a in (5, t.ca[1]):
        for i in (0, t.nx - 1):
            F = np.zeros((1, 14, t.nx))
            F[0, a, i] = 1.0
            O, _ = oracle.had(t, F)
            want = np.zeros(t.ndata)
            if (a, a) in pairs:
                want = t.fk[:, pairs.index((a, a)), i, i]
            assert np.array_equal(O[0], want)


def test_had_polarisation_recovers_offdiagonal_slice():
    """F = e_(a,i) + e_(b,j), a != b: O = FK[(a,a),i,i] + FK[(a,b),i,j]
    + FK[(b,a),j,i] + FK[(b,b),j,j] (absent channels count as 0)."""
    t = _had_float(seed=12)
    pairs = list(zip(t.ca.tolist(), t.cb.tolist()))
    a, b = pairs[2]
    if a == b:
        a, b = pairs[3]
    i, j = 1, 4

    def sl(p, u, v):
        return t.fk[:, pairs.index(p), u, v] if p in pairs else np.zeros(t.ndata)

    F = np.zeros((1, 14, t.nx))
    F[0, a, i] = 1.0
    F[0, b, j] = 1.0
    O, _ = oracle.had(t, F)
    want = sl((a, a), i, i) + sl((a, b), i, j) + sl((b, a), j, i) + sl((b, b), j, j)
    np.testing.assert_allclose(O[0], want, rtol=2e-16, atol=0)


def test_dis_delta_pdf_returns_slice():
    t, _ = W.config0()
    for a in range(14):
        F = np.zeros((1, 14, t.nx))
        F[0, a, 7] = 1.0
        O, _ = oracle.dis(t, F)
        assert np.array_equal(O[0], t.fk[:, a, 7])


# ------------------------------------------------ linearity / quadratic ----

def test_dis_linearity():
    t, F = W.config0()
    rng = np.random.default_rng(3)
    G = rng.uniform(0, 1, F.shape)
    O1, S1 = oracle.dis(t, F)
    O2, S2 = oracle.dis(t, G)
    O3, _ = oracle.dis(t, 0.75 * F - 1.5 * G)
    np.testing.assert_allclose(O3, 0.75 * O1 - 1.5 * O2, rtol=0, atol=1e-15 * (S1 + S2).max())
    O4, _ = oracle.dis(t, 2.0 * F)
    assert np.array_equal(O4, 2.0 * O1)


def test_had_homogeneity_and_parallelogram():
    t, F = W.config1(R=1, ndata=6, nc=9, nx=8)
    rng = np.random.default_rng(5)
    G = F * rng.uniform(0.5, 1.5, F.shape)
    O, S = oracle.had(t, F)
    O2, _ = oracle.had(t, 2.0 * F)
    assert np.array_equal(O2, 4.0 * O)  # power-of-two scaling is exact
    Op, Sp = oracle.had(t, F + G)
    Om, _ = oracle.had(t, F - G)
    Og, Sg = oracle.had(t, G)
    lhs = Op + Om
    rhs = 2.0 * O + 2.0 * Og
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-14 * (Sp + S + Sg).max())
    # the form is not symmetric in the table's i/j roles: transposing every
    # block without swapping the channel's flavours must change the result
    tt = T(t.fk.transpose(0, 1, 3, 2), t.xmap, t.nxg, t.ca, t.cb)
    Ot, _ = oracle.had(tt, F)
    assert np.abs(Ot - O).max() > 1e-6 * np.abs(O).max()


def test_had_flavour_swap_symmetry():
    """T^s[d,(b,a),j,i] = T[d,(a,b),i,j] gives the same observables, and the
    symmetrised table T + T^s gives twice them."""
    t, F = W.config1(R=3, ndata=5, nc=11, nx=7)
    ts = T(t.fk.transpose(0, 1, 3, 2).copy(), t.xmap, t.nxg, t.cb, t.ca)
    O, S = oracle.had(t, F)
    Os, _ = oracle.had(ts, F)
    np.testing.assert_allclose(Os, O, rtol=0, atol=1e-14 * S.max())
    both = T(np.concatenate([t.fk, ts.fk], axis=1), t.xmap, t.nxg,
             np.concatenate([t.ca, ts.ca]), np.concatenate([t.cb, ts.cb]))
    Ob, Sb = oracle.had(both, F)
    np.testing.assert_allclose(Ob, 2.0 * O, rtol=0, atol=1e-14 * Sb.max())


def test_had_separable_closed_form():
    """FK[d,c,i,j] = u_d v_c s_i t_j  =>  O[d] = u_d sum_c v_c (s . f_a)(t . f_b)."""
    rng = np.random.default_rng(9)
    nd, nc, nx, nxg = 4, 13, 9, 12
    u, v = rng.uniform(-1, 1, nd), rng.uniform(-1, 1, nc)
    s, tt = rng.uniform(0, 1, nx), rng.uniform(0, 1, nx)
    fk = u[:, None, None, None] * v[None, :, None, None] * s[None, None, :, None] * tt[None, None, None, :]
    ca, cb = W.channels(rng, nc)
    xmap = np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32)
    F = rng.uniform(0, 2, (2, 14, nxg))
    t = T(fk, xmap, nxg, ca, cb)
    O, S = oracle.had(t, F)
    Fx = F[:, :, xmap]
    for r in range(2):
        want = u * sum(v[c] * (s @ Fx[r, ca[c]]) * (tt @ Fx[r, cb[c]]) for c in range(nc))
        np.testing.assert_allclose(O[r], want, rtol=0, atol=1e-14 * S[r].max())
    # all-ones special case: sum_c Fbar_a Fbar_b
    t1 = T(np.ones((1, nc, nx, nx)), xmap, nxg, ca, cb)
    O1, _ = oracle.had(t1, F)
    Fb = Fx.sum(axis=2)
    for r in range(2):
        assert abs(O1[r, 0] - sum(Fb[r, ca[c]] * Fb[r, cb[c]] for c in range(nc))) < 1e-12 * abs(O1[r, 0])


# --------------------------------------------------------------- gradient ----

def test_had_grad_adjoint_identity_and_fd():
    t, F = W.config1(R=2, ndata=7, nc=10, nx=9)
    rng = np.random.default_rng(21)
    gO = rng.standard_normal((2, t.ndata))
    gF = oracle.had_grad(t, F, gO)
    dF = rng.standard_normal(F.shape) * F
    # quadratic form: J dF = (O(F+dF) - O(F-dF)) / 2 exactly up to rounding
    Op, Sp = oracle.had(t, F + dF)
    Om, Sm = oracle.had(t, F - dF)
    JdF = (Op - Om) / 2.0
    lhs = np.sum(gO * JdF)
    rhs = np.sum(gF * dF)
    scale = np.sum(np.abs(gO) * (Sp + Sm))
    assert abs(lhs - rhs) <= 1e-13 * scale
    # central finite differences, h = 1e-6 (absolute), on 12 coordinates
    h = 1e-6
    for _ in range(12):
        r, a, m = rng.integers(2), rng.integers(14), rng.integers(t.nxg)
        Fp, Fm = F.copy(), F.copy()
        Fp[r, a, m] += h
        Fm[r, a, m] -= h
        fd = np.sum(gO[r] * (oracle.had(t, Fp[r:r + 1])[0][0] - oracle.had(t, Fm[r:r + 1])[0][0])) / (2 * h)
        assert abs(fd - gF[r, a, m]) <= 1e-6 * max(abs(gF[r, a, m]), 1e-3 * np.abs(gF).max())


def test_had_grad_euler_identity():
    """Degree-2 homogeneity: sum F * dO/dF = 2 O for every (r, d)."""
    t, F = W.config1(R=2, ndata=4, nc=8, nx=6)
    O, S = oracle.had(t, F)
    for d in range(t.ndata):
        e = np.zeros((2, t.ndata))
        e[:, d] = 1.0
        g = oracle.had_grad(t, F, e)
        np.testing.assert_allclose((g * F).sum(axis=(1, 2)), 2 * O[:, d], rtol=0, atol=1e-13 * S[:, d].max())


def test_dis_grad_matches_delta_slices():
    t, F = W.config0()
    gO = np.zeros((1, t.ndata))
    gO[0, 3] = 1.0
    gF = oracle.dis_grad(t, gO)
    assert np.array_equal(gF[0], t.fk[3])


# ----------------------------------------------------------- chi^2 ----------

def _spd(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, min(n, 10)))
    return G @ G.T + np.diag(rng.uniform(0.1, 1.0, n))


@pytest.mark.parametrize("n", [1, 2, 17, 120])
def test_cholesky_reconstructs_and_matches_library(n):
    C = _spd(n, n)
    L = oracle.cholesky(C)
    assert np.allclose(np.triu(L, 1), 0)
    assert np.linalg.norm(L @ L.T - C) <= 1e-14 * np.linalg.norm(C)
    np.testing.assert_allclose(L, np.linalg.cholesky(C), rtol=1e-12, atol=1e-13)


def test_cholesky_rejects_non_spd():
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_chi2_special_cases_and_library():
    n, R = 60, 4
    C = _spd(n, 3)
    L = oracle.cholesky(C)
    rng = np.random.default_rng(4)
    D = rng.standard_normal(n)
    O = rng.standard_normal((R, n))
    c, g = oracle.chi2(L, O, D)
    for r in range(R):
        res = O[r] - D
        y = np.linalg.solve(C, res)
        assert abs(c[r] - res @ y) <= 1e-12 * abs(res @ y)
        np.testing.assert_allclose(g[r], 2 * y, rtol=1e-10, atol=1e-12 * np.abs(y).max())
    c0, g0 = oracle.chi2(L, np.tile(D, (2, 1)), D)
    assert np.all(c0 == 0) and np.all(g0 == 0)
    cI, gI = oracle.chi2(np.eye(n), O, D)
    np.testing.assert_allclose(cI, ((O - D) ** 2).sum(axis=1), rtol=1e-14)
    np.testing.assert_allclose(gI, 2 * (O - D), rtol=1e-15)


def test_chi2_gradient_is_exact_central_difference():
    """chi^2 is quadratic in O, so a central difference equals dchi2/dO."""
    n = 9
    C = _spd(n, 8)
    L = oracle.cholesky(C)
    rng = np.random.default_rng(8)
    D, O = rng.standard_normal(n), rng.standard_normal((1, n))
    _, g = oracle.chi2(L, O, D)
    for k in range(n):
        e = np.zeros((1, n))
        e[0, k] = 0.5
        fd = (oracle.chi2(L, O + e, D, False)[0] - oracle.chi2(L, O - e, D, False)[0]) / 1.0
        assert abs(fd[0] - g[0, k]) <= 1e-11 * np.abs(g).max()


# ------------------------------------------- dense product (Table 3) ----

def test_dense_exact_bruteforce():
    """The dense product of the paper's Table 3 on small integers, against a
    rational brute-force sum written from its definition."""
    rng = np.random.default_rng(11)
    nd, K, R = 4, 37, 3
    fk = rng.integers(-5, 6, (nd, K)).astype(np.float64)
    L = rng.integers(-5, 6, (R, K)).astype(np.float64)
    O, S = oracle.dense(fk, L)
    for r in range(R):
        for d in range(nd):
            want = sum(Fraction(int(fk[d, k])) * Fraction(int(L[r, k])) for k in range(K))
            assert O[r, d] == float(want)
            assert S[r, d] == float(sum(abs(Fraction(int(fk[d, k])) * Fraction(int(L[r, k]))) for k in range(K)))


def test_dense_one_hot_selects_columns():
    """A PDF matrix whose replica r is the unit vector e_{k_r} returns column
    k_r of the table: catches a transposed operand or a shifted index."""
    rng = np.random.default_rng(12)
    nd, K = 5, 23
    fk = rng.standard_normal((nd, K))
    ks = [0, 7, 22, 13]
    L = np.zeros((len(ks), K))
    for r, k in enumerate(ks):
        L[r, k] = 1.0
    O, _ = oracle.dense(fk, L)
    for r, k in enumerate(ks):
        assert np.array_equal(O[r], fk[:, k])


@pytest.mark.parametrize("seed", [1, 2])
def test_dense_of_luminosity_is_eq1_exactly(seed):
    """Table 3's formulation (flattened table times the PDF matrix) and Eq. 1
    (the per-channel quadratic form) are the same sum in different orders; on
    integer inputs both are exact, so they must agree bit for bit, and the
    PDF matrix must hold f_a(x_i) f_b(x_j) at element (c, i, j)."""
    t, F = _tiny_int_had(seed)
    L = oracle.luminosity(t, F)
    nc, nx = len(t.ca), len(t.xmap)
    r, c, i, j = 1, 2, 0, 2
    assert L[r, (c * nx + i) * nx + j] == F[r, t.ca[c], t.xmap[i]] * F[r, t.cb[c], t.xmap[j]]
    Od, Sd = oracle.dense(t.fk.reshape(t.fk.shape[0], -1), L)
    Oh, Sh = oracle.had(t, F)
    assert np.array_equal(Od, Oh) and np.array_equal(Sd, Sh)


def test_dense_of_luminosity_matches_eq1_on_config1():
    """Same identity on the config-1 table with real-valued PDFs: the two
    orders of summation agree within a few units of rounding of S."""
    t, F = W.config1(R=3)
    Od, Sd = oracle.dense(t.fk.reshape(t.fk.shape[0], -1), oracle.luminosity(t, F))
    Oh, Sh = oracle.had(t, F)
    assert np.abs(Od - Oh).max() <= 1e-15 * Sh.max()
