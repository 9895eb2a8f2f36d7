"""Pins for the oracle Poisson solve of the mean fields (Sec. 3.1, Eq. mean-field
and the Poisson equation with direct-integral boundary data)."""
import math

import numpy as np
import pytest
from scipy import special
from scipy.special import erf

from oracle import fem, mesh, poisson


@pytest.fixture(scope="module")
def h_q3():
    m = mesh.Mesh(-10.0, 10.0, 4, 3, [((0.0, 0.0, 0.0), 1.0, 3)], 2.0)
    op = fem.Operators(m)
    return m, op, poisson.PoissonSolver(op)


def test_real_harmonics_addition_theorem():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((20, 3))
    b = rng.standard_normal((20, 3))
    a /= np.linalg.norm(a, axis=1)[:, None]
    b /= np.linalg.norm(b, axis=1)[:, None]
    ta, pa = np.arccos(a[:, 2]), np.arctan2(a[:, 1], a[:, 0])
    tb, pb = np.arccos(b[:, 2]), np.arctan2(b[:, 1], b[:, 0])
    for l in range(poisson.LMAX + 1):
        s = sum(poisson.real_sph_harm(l, m_, ta, pa) * poisson.real_sph_harm(l, m_, tb, pb)
                for m_ in range(-l, l + 1))
        ref = (2 * l + 1) / (4 * math.pi) * special.eval_legendre(l, np.sum(a * b, axis=1))
        np.testing.assert_allclose(s, ref, atol=1e-12 * (2 * l + 1))


def test_real_harmonics_orthonormal():
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phi = 2 * np.pi * np.arange(nphi) / nphi
    T, P = np.meshgrid(np.arccos(xg), phi, indexing="ij")
    W = np.outer(wg, np.full(nphi, 2 * np.pi / nphi))
    idx = [(l, m_) for l in range(7) for m_ in range(-l, l + 1)]
    Y = np.array([poisson.real_sph_harm(l, m_, T, P).ravel() for (l, m_) in idx])
    G = (Y * W.ravel()) @ Y.T
    np.testing.assert_allclose(G, np.eye(len(idx)), atol=1e-12)


def test_multipole_matches_direct_sum_off_centre():
    """Boundary data from the l <= 12 expansion vs the literal direct integral
    (same quadrature) for an off-centre charge; truncation ~ (r'/r)^13."""
    m = mesh.Mesh(-8.0, 8.0, 4, 2, [((1.0, -0.5, 0.3), 1.0, 2)], 2.0)
    op = fem.Operators(m)
    ps = poisson.PoissonSolver(op)
    c0 = np.array([1.0, -0.5, 0.3])
    rho = np.exp(-2.0 * np.sum((m.X - c0) ** 2, axis=1))
    rho[np.any(np.isclose(np.abs(m.X), 8.0), axis=1)] = 0.0
    q = poisson.multipole_moments(m.X, op.m_f, rho[:, None], ps.center)
    sel = np.arange(0, len(ps.B), 7)
    g = poisson.multipole_potential(q, ps.Xb[sel], ps.center)[:, 0]
    gd = poisson.direct_potential(m.X, op.m_f, rho[:, None], ps.Xb[sel])[:, 0]
    assert np.abs(g - gd).max() < 1e-8 * np.abs(gd).max()
    # the monopole is the total charge
    assert abs(q[(0, 0)][0] * math.sqrt(4 * math.pi) - op.m_f @ rho) < 1e-13


def test_gaussian_charge_potential_and_self_energy(h_q3):
    """|phi|^2 with phi = e^{-r^2} normalised is a Gaussian of exponent 2:
    W = erf(sqrt2 r)/r and the self-energy int rho W = 2/sqrt(pi)."""
    m, op, ps = h_q3
    phi = np.exp(-np.sum(m.Xm ** 2, axis=1)) * (~m.boundary)
    phi /= math.sqrt(phi @ (op.ML * phi))
    rho, _ = poisson.pair_densities(op, phi[:, None].astype(complex))
    W = ps.solve(rho, method="cg", rtol=1e-12)[:, 0]
    r = np.linalg.norm(m.Xm, axis=1)
    a = math.sqrt(2.0)
    Wex = np.where(r > 0, erf(a * r) / np.where(r > 0, r, 1.0), 2 * a / math.sqrt(math.pi))
    assert np.abs(W - Wex).max() < 1e-3
    assert np.abs(W - Wex)[m.boundary].max() < 1e-9
    J = np.sum(op.m_f * rho[:, 0] * (op.C @ W))
    assert abs(J - 2 / math.sqrt(math.pi)) < 1e-4


def test_hydrogen_1s_hartree_potential(h_q3):
    """rho = e^{-2r}/pi gives W = 1/r - (1 + 1/r) e^{-2r}."""
    m, op, ps = h_q3
    phi = np.exp(-np.linalg.norm(m.Xm, axis=1)) * (~m.boundary)
    phi /= math.sqrt(phi @ (op.ML * phi))
    rho, _ = poisson.pair_densities(op, phi[:, None].astype(complex))
    W = ps.solve(rho, method="cg", rtol=1e-12)[:, 0]
    r = np.linalg.norm(m.Xm, axis=1)
    rs = np.where(r > 0, r, 1.0)
    Wex = np.where(r > 0, 1 / rs - (1 + 1 / rs) * np.exp(-2 * r), 1.0)
    assert np.abs(W - Wex).max() < 5e-3
    far = r > 3.0
    assert np.abs(W - Wex)[far].max() < 2e-4


def test_cg_matches_direct_and_pair_symmetry():
    m = mesh.Mesh(-6.0, 6.0, 3, 2, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)
    op = fem.Operators(m)
    ps = poisson.PoissonSolver(op)
    rng = np.random.default_rng(2)
    g1 = np.exp(-np.sum((m.Xm - [0, 0, 0.7]) ** 2, axis=1))
    g2 = np.exp(-0.7 * np.sum((m.Xm + [0.3, 0, 0.7]) ** 2, axis=1))
    phi = np.stack([g1 * np.exp(1j * rng.uniform(0, 0.3, m.N)), g2 * (1 + 0.2j)], axis=1)
    phi[m.boundary] = 0
    rho, pairs = poisson.pair_densities(op, phi)
    assert len(pairs) == 4
    Wd = ps.solve(rho, method="direct")
    Wc = ps.solve(rho, method="cg", rtol=1e-12)
    assert np.all(ps.residual(Wd, rho) < 1e-12)
    assert np.all(ps.residual(Wc, rho) < 1e-11)
    np.testing.assert_allclose(Wc, Wd, atol=1e-8 * np.abs(Wd).max())
    W = poisson.assemble_pair_potentials(Wd, pairs, 2)
    np.testing.assert_array_equal(W[1, 0], np.conj(W[0, 1]))
    # linearity: W_01 is the potential of conj(phi_0) phi_1 as one complex density
    z = np.conj(op.C @ phi[:, 0]) * (op.C @ phi[:, 1])
    Wre = ps.solve(z.real[:, None], method="direct")[:, 0]
    Wim = ps.solve(z.imag[:, None], method="direct")[:, 0]
    np.testing.assert_allclose(W[0, 1], Wre + 1j * Wim, atol=1e-12 * np.abs(Wre).max())
