"""Randomised properties of the oracle (CPU, bounded example counts).

The pins in test_oracle_pins.py use fixed small cases; these draw shapes,
channel lists, grids and values at random and check identities that hold
for any input, so an index or layout mistake that a fixed case misses still
shows up:
  * Eq. 1 is a quadratic form: O(λ f) = λ² O(f), and with integer inputs the
    oracle equals a rational brute force;
  * the flattened dense product with the PDF matrix equals Eq. 1 (Table 3's
    formulation and the per-channel quadratic form are one sum);
  * DIS observables are linear in f;
  * the adjoint satisfies <gO, dO/df · v> = <gF, v> for the hadronic form,
    checked through the exact central difference of a quadratic.
"""
from fractions import Fraction

import numpy as np
from hypothesis import HealthCheck, given, settings, strategies as st

import oracle


class T:
    def __init__(self, fk, xmap, nxg, ca=None, cb=None):
        self.fk = np.asarray(fk, np.float64)
        self.xmap = np.asarray(xmap, np.int32)
        self.nxg = nxg
        if ca is not None:
            self.ca = np.asarray(ca, np.int32)
            self.cb = np.asarray(cb, np.int32)


@st.composite
def had_case(draw, max_nd=3, max_nc=4, max_nx=4, max_R=3):
    nd = draw(st.integers(1, max_nd))
    nc = draw(st.integers(1, max_nc))
    nx = draw(st.integers(1, max_nx))
    nxg = draw(st.integers(nx, nx + 3))
    R = draw(st.integers(1, max_R))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    pairs = rng.choice(196, nc, replace=False)
    ca, cb = pairs // 14, pairs % 14
    xmap = np.sort(rng.choice(nxg, nx, replace=False))
    fk = rng.integers(-3, 4, (nd, nc, nx, nx)).astype(np.float64)
    F = rng.integers(-3, 4, (R, 14, nxg)).astype(np.float64)
    return T(fk, xmap, nxg, ca, cb), F


SETTINGS = settings(max_examples=40, deadline=None, suppress_health_check=[HealthCheck.too_slow])


@SETTINGS
@given(had_case())
def test_eq1_matches_rational_bruteforce_and_is_quadratic(case):
    t, F = case
    O, S = oracle.had(t, F)
    for r in range(F.shape[0]):
        for d in range(t.fk.shape[0]):
            want = Fraction(0)
            for c in range(len(t.ca)):
                for i in range(len(t.xmap)):
                    for j in range(len(t.xmap)):
                        want += (Fraction(int(t.fk[d, c, i, j])) * int(F[r, t.ca[c], t.xmap[i]])
                                 * int(F[r, t.cb[c], t.xmap[j]]))
            assert O[r, d] == float(want)
    O3, _ = oracle.had(t, 3.0 * F)
    assert np.array_equal(O3, 9.0 * O)
    assert np.all(S >= np.abs(O))


@SETTINGS
@given(had_case(max_nd=4, max_nc=6, max_nx=5, max_R=4))
def test_dense_product_of_pdf_matrix_is_eq1(case):
    t, F = case
    L = oracle.luminosity(t, F)
    Od, Sd = oracle.dense(t.fk.reshape(t.fk.shape[0], -1), L)
    Oh, Sh = oracle.had(t, F)
    assert np.array_equal(Od, Oh) and np.array_equal(Sd, Sh)


@SETTINGS
@given(st.integers(1, 4), st.integers(1, 6), st.integers(0, 3), st.integers(0, 2 ** 31 - 1))
def test_dis_is_linear(nd, nx, extra, seed):
    rng = np.random.default_rng(seed)
    nxg = nx + extra
    xmap = np.sort(rng.choice(nxg, nx, replace=False))
    t = T(rng.integers(-3, 4, (nd, 14, nx)), xmap, nxg)
    f = rng.integers(-3, 4, (2, 14, nxg)).astype(np.float64)
    g = rng.integers(-3, 4, (2, 14, nxg)).astype(np.float64)
    Of, _ = oracle.dis(t, f)
    Og, _ = oracle.dis(t, g)
    Ofg, _ = oracle.dis(t, 2.0 * f - 3.0 * g)
    assert np.array_equal(Ofg, 2.0 * Of - 3.0 * Og)


@SETTINGS
@given(had_case(max_R=2))
def test_had_adjoint_matches_exact_directional_difference(case):
    """Eq. 1 is quadratic, so (O(f + v) - O(f - v)) / 2 is exactly dO/df · v
    for any step v; contracted with gO it must equal <gF, v>."""
    t, F = case
    rng = np.random.default_rng(int(abs(F).sum()) + 7)
    gO = rng.integers(-3, 4, (F.shape[0], t.fk.shape[0])).astype(np.float64)
    v = rng.integers(-2, 3, F.shape).astype(np.float64)
    gF = oracle.had_grad(t, F, gO)
    Op, _ = oracle.had(t, F + v)
    Om, _ = oracle.had(t, F - v)
    lhs = (gO * (Op - Om) / 2.0).sum()
    assert lhs == (gF * v).sum()
