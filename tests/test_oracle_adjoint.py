"""Pins of the oracle's dense adjoint and tangent of the one-electron step
(Sec. 3.2 with one orbital; Sec. 3.1 operators) against facts that do not
come from the oracle itself: central finite differences of the forward map,
the dot-product identity between tangent and adjoint, M_L-norm conservation
(the propagator is unitary in <.,.>_M), and the closed form of the first
step's response from an eigenstate via the eigen-decomposition."""
import numpy as np
import pytest
import scipy.linalg

from oracle import adjoint, fem, mesh as omesh
from paper_2301_02387_gb300 import inputs

CASE = (-6.0, 6.0, 3, 2, [((0.5, 0.5, 0.7), 1.0, 1), ((0.5, 0.5, -0.7), 1.0, 1)], 0.5)


@pytest.fixture(scope="module")
def sys1():
    om = omesh.Mesh(*CASE)
    op = fem.Operators(om)
    td = adjoint.TDSE(op, e_dir=(0.0, 0.0, 1.0))
    phi = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, CASE[4], 1), op.ML)[:, 0]
    return td, td.restrict(phi)


def _fields(K, seed):
    rng = np.random.default_rng(seed)
    return 0.05 * rng.standard_normal(K)


def test_gradient_matches_central_differences(sys1):
    td, phi0 = sys1
    K, dt = 5, 0.1
    E = _fields(K, 1)
    g = np.random.default_rng(2).standard_normal(K + 1)
    grad, _ = td.vjp(phi0, E, dt, g)
    h = 1e-6
    fd = np.zeros(K)
    for k in range(K):
        Ep, Em = E.copy(), E.copy()
        Ep[k] += h
        Em[k] -= h
        fd[k] = (g @ td.forward(phi0, Ep, dt)[0] - g @ td.forward(phi0, Em, dt)[0]) / (2 * h)
    assert np.max(np.abs(grad - fd)) <= 1e-7 * np.max(np.abs(fd))


def test_tangent_matches_central_differences(sys1):
    td, phi0 = sys1
    K, dt = 4, 0.1
    E = _fields(K, 3)
    v = np.random.default_rng(4).standard_normal(K)
    d, dd = td.jvp(phi0, E, dt, v)
    h = 1e-6
    fd = (td.forward(phi0, E + h * v, dt)[0] - td.forward(phi0, E - h * v, dt)[0]) / (2 * h)
    np.testing.assert_allclose(d, td.forward(phi0, E, dt)[0], rtol=0, atol=1e-14)
    assert dd[0] == 0.0
    assert np.max(np.abs(dd - fd)) <= 1e-7 * np.max(np.abs(fd))


def test_dot_product_identity(sys1):
    td, phi0 = sys1
    K, dt = 6, 0.1
    E = _fields(K, 5)
    rng = np.random.default_rng(6)
    v = rng.standard_normal(K)
    g = rng.standard_normal(K + 1)
    _, dd = td.jvp(phi0, E, dt, v)
    grad, _ = td.vjp(phi0, E, dt, g)
    lhs, rhs = g @ dd, v @ grad
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs))


def test_norm_conserved(sys1):
    td, phi0 = sys1
    _, phis = td.forward(phi0, _fields(8, 7), 0.1)
    norms = np.array([td.inner(p, p).real for p in phis])
    np.testing.assert_allclose(norms, 1.0, rtol=0, atol=1e-12)


def test_eigenstate_first_step_closed_form(sys1):
    """From a discrete eigenstate psi_0 of H~(0) with E = 0, d_0 = d_1 and
    dd_1/dE_0 = -2 sum_n |Z_n0|^2 (1 - cos(dt w_n)) / w_n, w_n = eps_n - eps_0,
    Z_n0 = psi_n^H F psi_0 (M-orthonormal eigenvectors)."""
    td, _ = sys1
    eps, Psi = scipy.linalg.eigh(td.H0, np.diag(td.m))
    psi0 = Psi[:, 0].astype(np.complex128)
    dt = 0.2
    d, _ = td.forward(psi0, np.zeros(1), dt)
    assert abs(d[1] - d[0]) <= 1e-12 * max(1.0, abs(d[0]))
    Z = Psi.T @ (td.F @ Psi[:, 0])
    w = eps - eps[0]
    terms = np.zeros_like(w)
    nz = np.abs(w) > 1e-12
    terms[nz] = np.abs(Z[nz]) ** 2 * (1.0 - np.cos(dt * w[nz])) / w[nz]
    expect = -2.0 * terms.sum()
    grad, _ = td.vjp(psi0, np.zeros(1), dt, np.array([0.0, 1.0]))
    assert abs(grad[0] - expect) <= 1e-10 * abs(expect)
    _, dd = td.jvp(psi0, np.zeros(1), dt, np.ones(1))
    assert abs(dd[1] - expect) <= 1e-10 * abs(expect)


def test_adjoint_state_is_gradient_wrt_initial_state(sys1):
    """lam_0 is the M-gradient of J = g.d with respect to phi_0:
    dJ = 2 Re <lam_0, dphi_0>_M for a perturbation dphi_0."""
    td, phi0 = sys1
    K, dt = 3, 0.1
    E = _fields(K, 8)
    g = np.random.default_rng(9).standard_normal(K + 1)
    _, lam0 = td.vjp(phi0, E, dt, g)
    rng = np.random.default_rng(10)
    dphi = rng.standard_normal(phi0.shape) + 1j * rng.standard_normal(phi0.shape)
    h = 1e-6
    fd = (g @ td.forward(phi0 + h * dphi, E, dt)[0] - g @ td.forward(phi0 - h * dphi, E, dt)[0]) / (2 * h)
    pred = 2.0 * np.real(td.inner(lam0, dphi))
    assert abs(pred - fd) <= 1e-7 * abs(fd)


@pytest.fixture(scope="module")
def sys_force():
    om = omesh.Mesh(*CASE)
    op = fem.Operators(om)
    td = adjoint.TDSE(op, e_dir=(0.3, -0.4, 0.866), observable="force")
    phi = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, CASE[4], 1), op.ML)[:, 0]
    return td, td.restrict(phi)


def test_nuclear_force_is_minus_grad_potential():
    """f = -grad V against central differences of the oracle's potential at the
    support points (those at least 0.3 bohr from every nucleus)."""
    om = omesh.Mesh(*CASE)
    op = fem.Operators(om)
    X = om.X
    F = op.nuclear_force(X)
    far = np.ones(len(X), dtype=bool)
    for (R, _Z, _L) in om.nuclei:
        far &= np.linalg.norm(X - R[None, :], axis=1) > 0.3
    assert far.sum() > 100
    h = 1e-5
    for k in range(3):
        dX = np.zeros(3)
        dX[k] = h
        fd = -(op.nuclear_potential(X + dX) - op.nuclear_potential(X - dX)) / (2 * h)
        np.testing.assert_allclose(F[far, k], fd[far], rtol=1e-6, atol=1e-8)
    on = np.zeros(len(X), dtype=bool)
    for (R, _Z, _L) in om.nuclei:
        on |= np.linalg.norm(X - R[None, :], axis=1) < 1e-10
    assert np.all(F[on] == 0.0)


def test_force_observable_gradient_and_dot_product(sys_force):
    """The adjoint with the force signal: central differences and the
    dot-product identity, as for the dipole."""
    td, phi0 = sys_force
    K, dt = 4, 0.1
    E = _fields(K, 21)
    rng = np.random.default_rng(22)
    g = rng.standard_normal(K + 1)
    v = rng.standard_normal(K)
    grad, _ = td.vjp(phi0, E, dt, g)
    _, dd = td.jvp(phi0, E, dt, v)
    assert abs(g @ dd - v @ grad) <= 1e-10 * max(abs(g @ dd), abs(v @ grad))
    h = 1e-6
    fd = np.zeros(K)
    for k in range(K):
        Ep, Em = E.copy(), E.copy()
        Ep[k] += h
        Em[k] -= h
        fd[k] = (g @ td.forward(phi0, Ep, dt)[0] - g @ td.forward(phi0, Em, dt)[0]) / (2 * h)
    assert np.max(np.abs(grad - fd)) <= 1e-7 * np.max(np.abs(fd))
