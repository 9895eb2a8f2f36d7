"""Gauss-Lobatto-Legendre (GLL) nodes, weights and the 1D Lagrange basis on [0, 1].

Sec. 3.1: the cell basis functions are products of 1D Lagrange polynomials
through the GLL points, and every integral uses GLL quadrature on the same
points (the FEDVR construction).  Here the reference interval is [0, 1].

Test infrastructure only (see the package docstring).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gll_nodes_weights(p):
    """Return (xi, w): the p+1 GLL nodes on [0,1] (ascending) and their weights.

    On [-1,1] the nodes are the endpoints and the roots of P_p'(x); the weights
    are 2 / (p (p+1) P_p(x_i)^2).  The affine map to [0,1] halves the weights.
    """
    if p < 1:
        raise ValueError("degree must be >= 1")
    cp = np.zeros(p + 1)
    cp[p] = 1.0                      # Legendre-series coefficients of P_p
    if p == 1:
        interior = np.zeros(0)
    else:
        interior = np.sort(np.real(npleg.legroots(npleg.legder(cp))))
    x = np.concatenate(([-1.0], interior, [1.0]))
    Pp = npleg.legval(x, cp)
    w = 2.0 / (p * (p + 1) * Pp ** 2)
    return (x + 1.0) / 2.0, w / 2.0


def lagrange_matrix(nodes, x):
    """L[q, j] = L_j(x_q): the Lagrange polynomials through `nodes` evaluated at x."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_deriv_matrix(nodes, x):
    """D[q, j] = L_j'(x_q), by the product rule on the Lagrange product form."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[k]))
            for m in range(n):
                if m != j and m != k:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            D[:, j] += term
    return D


def stiffness_1d(p):
    """Khat[i, j] = sum_q w_q L_i'(xi_q) L_j'(xi_q) on [0,1] (GLL quadrature).

    L_i' L_j' has degree 2p-2 <= 2p-1, so the GLL rule makes this the exact
    1D stiffness matrix of the degree-p Lagrange basis.
    """
    xi, w = gll_nodes_weights(p)
    D = lagrange_deriv_matrix(xi, xi)
    return D.T @ np.diag(w) @ D
