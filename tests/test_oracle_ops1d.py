"""Pins for the oracle's 1-D operators (Sec. 2.1, FR divergence equation).

Every check compares against something other than the oracle itself: closed
forms, numpy's Gauss-Legendre and Legendre-series routines, polynomial
calculus, and the classical equivalence of FR with the DG correction to
nodal DG on Gauss points (Huynh 2007).
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

from oracle import ops1d


def test_gauss_closed_forms():
    x, w = ops1d.gauss_legendre(2)
    np.testing.assert_allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [1.0, 1.0], rtol=0, atol=1e-15)
    x, w = ops1d.gauss_legendre(3)
    np.testing.assert_allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], rtol=0, atol=1e-15)


@pytest.mark.parametrize("m", range(1, 10))
def test_gauss_matches_numpy(m):
    x, w = ops1d.gauss_legendre(m)
    xr, wr = npleg.leggauss(m)
    np.testing.assert_allclose(x, xr, rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, wr, rtol=0, atol=2e-15)


@pytest.mark.parametrize("m", range(1, 9))
def test_gauss_exact_to_degree_2m_minus_1(m):
    x, w = ops1d.gauss_legendre(m)
    for k in range(2 * m):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p", range(0, 7))
def test_interpolation_and_derivative_exact(p):
    m = p + 1
    x, _ = ops1d.gauss_legendre(m)
    rng = np.random.default_rng(p)
    coef = rng.normal(size=m)              # random polynomial of degree p
    f = nppoly.polyval(x, coef)
    xs = np.concatenate([[-1.0, 1.0], rng.uniform(-1, 1, 5)])
    L = ops1d.lagrange(x, xs)
    np.testing.assert_allclose(L @ f, nppoly.polyval(xs, coef), rtol=0, atol=1e-12)
    D = ops1d.lagrange_deriv(x, x)
    np.testing.assert_allclose(D @ f, nppoly.polyval(x, nppoly.polyder(coef)), rtol=0, atol=1e-11)
    # derivative at arbitrary points as well
    Dx = ops1d.lagrange_deriv(x, xs)
    np.testing.assert_allclose(Dx @ f, nppoly.polyval(xs, nppoly.polyder(coef)), rtol=0, atol=1e-11)


@pytest.mark.parametrize("kind", ["dg", "g2"])
@pytest.mark.parametrize("m", range(2, 8))
def test_correction_endpoint_conditions(kind, m):
    hl, _ = ops1d.correction_left(kind, m, np.array([-1.0, 1.0]))
    hr, _ = ops1d.correction_right(kind, m, np.array([-1.0, 1.0]))
    np.testing.assert_allclose(hl, [1.0, 0.0], atol=1e-14)
    np.testing.assert_allclose(hr, [0.0, 1.0], atol=1e-14)


def _as_power_series(kind, m):
    """Fit h_l (degree m) exactly from m + 1 samples into a power series."""
    xs = np.cos(np.pi * (np.arange(m + 1) + 0.5) / (m + 1))
    h, _ = ops1d.correction_left(kind, m, xs)
    return nppoly.polyfit(xs, h, m)


@pytest.mark.parametrize("m", range(2, 8))
def test_dg_correction_is_right_radau(m):
    """h_l = R_{R,m} is the unique degree-m polynomial with h(-1) = 1, h(1) = 0,
    orthogonal to all polynomials of degree <= m - 2."""
    c = _as_power_series("dg", m)
    leg = npleg.poly2leg(c)
    assert np.all(np.abs(leg[: m - 1]) < 1e-12)      # orthogonal to P_0..P_{m-2}
    assert abs(nppoly.polyval(-1.0, c) - 1.0) < 1e-12
    assert abs(nppoly.polyval(1.0, c)) < 1e-12


@pytest.mark.parametrize("m", range(2, 8))
def test_g2_correction_defining_properties(m):
    """g2: degree m, h(-1) = 1, double root at +1, orthogonal to degree <= m - 3."""
    c = _as_power_series("g2", m)
    leg = npleg.poly2leg(c)
    if m >= 3:
        assert np.all(np.abs(leg[: m - 2]) < 1e-12)
    assert abs(nppoly.polyval(1.0, c)) < 1e-12
    assert abs(nppoly.polyval(1.0, nppoly.polyder(c))) < 1e-11
    assert abs(nppoly.polyval(-1.0, c) - 1.0) < 1e-12


@pytest.mark.parametrize("m", range(1, 8))
def test_dg_correction_recovers_nodal_dg_lifting(m):
    """FR with the DG correction on Gauss points is nodal DG with a diagonal
    mass matrix: h_l'(x_j) = -l_j(-1) / w_j and h_r'(x_j) = l_j(1) / w_j."""
    if m == 1:
        pytest.skip("p = 0 has no interior derivative")
    ops = ops1d.Ops1D(m - 1, "dg")
    np.testing.assert_allclose(ops.dhl, -ops.lm / ops.w, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ops.dhr, ops.lp / ops.w, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m", range(2, 8))
def test_correction_derivative_matches_series(m):
    for kind in ("dg", "g2"):
        c = _as_power_series(kind, m)
        xs = np.linspace(-0.9, 0.9, 7)
        _, dh = ops1d.correction_left(kind, m, xs)
        np.testing.assert_allclose(dh, nppoly.polyval(xs, nppoly.polyder(c)), atol=1e-10)
