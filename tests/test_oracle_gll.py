"""Pins for the oracle's GLL basis (Sec. 3.1: Lagrange polynomials through the
Gauss-Lobatto points, integrals by Gauss-Lobatto quadrature)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import gll

# Textbook Gauss-Lobatto rules on [-1, 1], mapped here to [0, 1] by (x+1)/2, w/2.
CLOSED = {
    1: ([-1.0, 1.0], [1.0, 1.0]),
    2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1.0, -1 / np.sqrt(5), 1 / np.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1.0, -np.sqrt(3 / 7), 0.0, np.sqrt(3 / 7), 1.0],
        [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_nodes_weights_closed_form(p):
    xi, w = gll.gll_nodes_weights(p)
    x_ref, w_ref = CLOSED[p]
    np.testing.assert_allclose(xi, (np.array(x_ref) + 1) / 2, atol=1e-15)
    np.testing.assert_allclose(w, np.array(w_ref) / 2, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_exact_to_degree_2p_minus_1_only(p):
    xi, w = gll.gll_nodes_weights(p)
    for k in range(2 * p):
        assert abs(np.dot(w, xi ** k) - 1.0 / (k + 1)) < 1e-14
    # a Lobatto rule with p+1 points is not exact at degree 2p
    assert abs(np.dot(w, xi ** (2 * p)) - 1.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_cardinal_and_derivative(p):
    xi, _ = gll.gll_nodes_weights(p)
    np.testing.assert_allclose(gll.lagrange_matrix(xi, xi), np.eye(p + 1), atol=1e-14)
    x = np.linspace(0.03, 0.97, 11)
    eps = 1e-6
    fd = (gll.lagrange_matrix(xi, x + eps) - gll.lagrange_matrix(xi, x - eps)) / (2 * eps)
    np.testing.assert_allclose(gll.lagrange_deriv_matrix(xi, x), fd, atol=1e-7)
    # partition of unity
    np.testing.assert_allclose(gll.lagrange_matrix(xi, x).sum(axis=1), 1.0, atol=1e-14)


def test_stiffness_p1_p2_closed_form():
    np.testing.assert_allclose(gll.stiffness_1d(1), [[1, -1], [-1, 1]], atol=1e-14)
    K2 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0
    np.testing.assert_allclose(gll.stiffness_1d(2), K2, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_stiffness_matches_gauss_legendre_integration(p):
    """int_0^1 L_i' L_j' by a 20-point Gauss-Legendre rule (numpy) agrees."""
    xi, _ = gll.gll_nodes_weights(p)
    xg, wg = npleg.leggauss(20)
    xg, wg = (xg + 1) / 2, wg / 2
    D = gll.lagrange_deriv_matrix(xi, xg)
    K = D.T @ np.diag(wg) @ D
    np.testing.assert_allclose(gll.stiffness_1d(p), K, atol=1e-12)
    np.testing.assert_allclose(gll.stiffness_1d(p).sum(axis=1), 0.0, atol=1e-12)
