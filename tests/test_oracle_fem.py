"""Pins for the oracle's assembled operators (Sec. 3.1): lumped mass,
stiffness, pointwise potentials and the one-body Hamiltonian matrix."""
import itertools

import numpy as np
import pytest

from oracle import fem, mesh

OFF_CASE = dict(lo=-8.0, hi=8.0, nc=4, nuclei=[((0.3, -0.45, 0.7), 1.0, 2),
                                             ((-1.1, 0.2, -0.35), 2.0, 3)], c=1.5)


def _ops(p, case=OFF_CASE):
    m = mesh.Mesh(case["lo"], case["hi"], case["nc"], p, case["nuclei"], case["c"])
    return m, fem.Operators(m)


def test_cube_mean_inverse_distance_constant():
    """c3 = mean of 1/|r| over the unit cube, by brute-force midpoint sums."""
    n = 120
    g = (np.arange(n) + 0.5) / n - 0.5
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    approx = np.mean(1.0 / np.sqrt(x * x + y * y + z * z))
    assert abs(approx - fem.CUBE_MEAN_INV_R) < 2e-3
    assert abs(fem.CUBE_MEAN_INV_R - 2.3800774) < 1e-7


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lumped_mass_integrates_q_p_polynomials_exactly(p):
    m, op = _ops(p)
    assert abs(op.ML.sum() - 16.0 ** 3) < 1e-9
    assert np.all(op.ML > 0)
    x, y, z = (m.Xm[:, a] for a in range(3))
    for a, b, c in [(1, 0, 0), (0, min(p, 2), 1), (p, p, p), (p, 0, p)]:
        exact = np.prod([(8.0 ** (k + 1) - (-8.0) ** (k + 1)) / (k + 1) for k in (a, b, c)])
        g = x ** a * y ** b * z ** c
        approx = np.dot(op.ML, g)
        assert abs(approx - exact) < 1e-13 * np.dot(op.ML, np.abs(g))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_stiffness_identities(p):
    """A 1 = 0; A x = 0 at interior masters; for p >= 2 also A (x y) = 0 and
    A x^2 = -2 M_L there (the functions lie in Q_p and GLL quadrature integrates
    these pairs exactly); A symmetric."""
    m, op = _ops(p)
    A = op.A
    x, y, z = (m.Xm[:, a] for a in range(3))
    I = ~m.boundary
    assert np.abs(A @ np.ones(m.N)).max() < 1e-11
    for f in (x, y, z):
        assert np.abs((A @ f)[I]).max() < 1e-10
    assert abs(A - A.T).max() < 1e-13
    if p == 1:
        return
    for f in (x * y, y * z):
        assert np.abs((A @ f)[I]).max() < 1e-10
    for f in (x * x, y * y, z * z):
        np.testing.assert_allclose((A @ f)[I], -2.0 * op.ML[I], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose((A @ (x * x + y * y - 2 * z * z))[I], 0.0, atol=1e-10)


def test_dipole_term_sign_and_axis():
    """<x_a> of a displaced Gaussian through F[E . x] equals its centre."""
    m, op = _ops(3)
    c0 = np.array([0.8, -0.5, 0.3])
    psi = np.exp(-np.sum((m.Xm - c0) ** 2, axis=1)) * (~m.boundary)
    norm = psi @ (op.ML * psi)
    H0 = op.H1_matrix()
    for ax in range(3):
        E = np.zeros(3)
        E[ax] = 1.0
        mom = psi @ ((op.H1_matrix(E) - H0) @ psi) / norm
        assert abs(mom - c0[ax]) < 1e-3


@pytest.mark.parametrize("L,p", [(2, 2), (3, 2), (4, 2)])
def test_hydrogen_rayleigh_quotient_h_convergence(L, p):
    """Rayleigh quotient of the exact 1s orbital e^-r approaches -1/2 Eh as the
    mesh is refined toward the nucleus (error bounds from the refinement study)."""
    bound = {2: 0.08, 3: 0.035, 4: 0.011}[L]
    m = mesh.Mesh(-10.0, 10.0, 4, p, [((0.0, 0.0, 0.0), 1.0, L)], 2.0)
    op = fem.Operators(m)
    psi = np.exp(-np.linalg.norm(m.Xm, axis=1)) * (~m.boundary)
    E = psi @ (op.H1_matrix() @ psi) / (psi @ (op.ML * psi))
    assert -0.5 < E < -0.5 + bound


def test_hydrogen_rayleigh_quotient_p_convergence():
    errs = []
    for p in (2, 3, 4):
        m = mesh.Mesh(-10.0, 10.0, 4, p, [((0.0, 0.0, 0.0), 1.0, 3)], 2.0)
        op = fem.Operators(m)
        psi = np.exp(-np.linalg.norm(m.Xm, axis=1)) * (~m.boundary)
        errs.append(psi @ (op.H1_matrix() @ psi) / (psi @ (op.ML * psi)) + 0.5)
    assert errs[0] > errs[1] > errs[2] > 0.0
    assert errs[2] < 0.005


def test_h1_apply_masks_boundary():
    m, op = _ops(2)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((m.N, 2)) + 1j * rng.standard_normal((m.N, 2))
    y = op.h1_apply(x, E=(0.01, 0.0, -0.02))
    assert np.all(y[m.boundary] == 0)
    x2 = x.copy()
    x2[m.boundary] = 0
    np.testing.assert_array_equal(op.h1_apply(x2, E=(0.01, 0.0, -0.02)), y)


# ------------------------------------------------------------- velocity gauge
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gradient_matrices_identities(p):
    """G_d (skew form of int b_k d_d b_l) is antisymmetric on the hanging-node
    mesh, so -i A.G is Hermitian.  On a conforming mesh, at interior masters
    whose support avoids the surface: G_x x = M_L and G_x y = 0, and for
    p >= 2 G_x x^2 = 2 x M_L (GLL quadrature is exact for these degrees)."""
    m, op = _ops(p)
    for d in range(3):
        G = op.gradient(d)
        assert abs(G + G.T).max() < 1e-13 * abs(G).max()
    mc, oc = _ops(p, dict(lo=-8.0, hi=8.0, nc=4, nuclei=[((0.3, -0.45, 0.7), 1.0, 0)], c=1.5))
    assert mc.n_hanging == 0
    deep = np.all(np.abs(mc.Xm) < 8.0 - 4.0 - 1e-9, axis=1)
    for d in range(3):
        G = oc.gradient(d)
        xd, xo = mc.Xm[:, d], mc.Xm[:, (d + 1) % 3]
        np.testing.assert_allclose((G @ xd)[deep], oc.ML[deep], rtol=1e-10, atol=0)
        assert np.max(np.abs((G @ xo)[deep])) < 1e-10 * np.max(oc.ML)
        if p >= 2:
            np.testing.assert_allclose((G @ xd ** 2)[deep], 2.0 * xd[deep] * oc.ML[deep], rtol=1e-10,
                                       atol=1e-10 * np.max(np.abs(xd) * oc.ML))


def test_velocity_gauge_hamiltonian_is_hermitian_and_gauge_consistent():
    """H1~(A) = 1/2 A + F[V] - i sum A_d G_d is Hermitian on the interior and
    its expectation in a real orbital equals the field-free one (the
    velocity term of a real function has zero expectation: antisymmetry)."""
    m, op = _ops(3)
    I = np.nonzero(~m.boundary)[0]
    A = (0.03, -0.05, 0.08)
    H = op.H1_matrix(A=A)[I][:, I]
    assert abs(H - H.conj().T).max() < 1e-13 * abs(H).max()
    rng = np.random.default_rng(2)
    u = rng.standard_normal(len(I))
    e0 = u @ (op.H1_matrix()[I][:, I] @ u)
    eA = np.vdot(u, H @ u)
    assert abs(eA.imag) < 1e-12 * abs(e0) and abs(eA.real - e0) < 1e-12 * abs(e0)


def test_velocity_term_measures_momentum():
    """Sign and factor of the velocity term: for u = exp(i k . x) g(x) with a
    smooth real envelope g, <u, -i G_d u> / <u, M_L u> = k_d + O(h^p) (the
    momentum of the plane wave; the envelope's own momentum is zero)."""
    m, op = _ops(4, dict(lo=-8.0, hi=8.0, nc=6, nuclei=[((0.0, 0.0, 0.0), 1.0, 1)], c=1.5))
    k = np.array([0.7, -0.4, 0.25])
    g = np.exp(-0.15 * np.sum(m.Xm ** 2, axis=1))
    u = g * np.exp(1j * (m.Xm @ k))
    u[m.boundary] = 0.0
    norm = np.vdot(u, op.ML * u).real
    for d in range(3):
        pd = np.vdot(u, -1j * (op.gradient(d) @ u)) / norm
        assert abs(pd.imag) < 1e-12 and abs(pd.real - k[d]) < 2e-3, (d, pd)
