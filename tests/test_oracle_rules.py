"""Pins for the oracle's 1D rules: Gauss-Legendre points and weights against
numpy's library routine and exactness on monomials; Gauss-Lobatto nodes against
their closed forms (the roots of P_p' plus the end points)."""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("q", range(1, 10))
def test_gauss_legendre_matches_numpy(q):
    xg, wg, _ = oracle.rules(1, q)
    xr, wr = np.polynomial.legendre.leggauss(q)
    np.testing.assert_allclose(xg, xr, atol=1e-15, rtol=0)
    np.testing.assert_allclose(wg, wr, atol=1e-15, rtol=0)


@pytest.mark.parametrize("q", range(1, 9))
def test_gauss_legendre_exact_to_degree_2q_minus_1(q):
    xg, wg, _ = oracle.rules(1, q)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(wg, xg ** k) - exact) < 1e-14


GLL_CLOSED = {
    1: [-1.0, 1.0],
    2: [-1.0, 0.0, 1.0],
    3: [-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0],
    4: [-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0],
    5: [-1.0, -math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21), -math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21),
        math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21), math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21), 1.0],
}


@pytest.mark.parametrize("p", sorted(GLL_CLOSED))
def test_gauss_lobatto_closed_forms(p):
    _, _, xn = oracle.rules(p, p + 2)
    np.testing.assert_allclose(xn, GLL_CLOSED[p], atol=1e-15, rtol=0)


@pytest.mark.parametrize("p", range(6, 9))
def test_gauss_lobatto_are_roots_of_legendre_derivative(p):
    _, _, xn = oracle.rules(p, p + 2)
    dP = np.polynomial.legendre.Legendre.basis(p).deriv()
    assert np.all(np.abs(dP(xn[1:-1])) < 1e-12)
    assert xn[0] == -1.0 and xn[-1] == 1.0 and np.all(np.diff(xn) > 0)
