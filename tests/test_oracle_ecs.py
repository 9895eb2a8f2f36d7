"""Oracle pins of exterior complex scaling (Sec. 4's absorbing boundary; the
reading is stated in ``oracle.fem``): the scaled operator reduces to the
unscaled one where nothing is scaled, its stiffness is complex symmetric,
the free kinetic operator's spectrum lies in the lower half plane (every mode
decays), and an outgoing free wave packet leaves the inner box as the exact
free solution does, where a hard wall reflects it."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from oracle import fem, mctdhf, mesh as omesh
from paper_2301_02387_gb300 import inputs

FREE = (-10.0, 10.0, 10, 3, [((0.0, 0.0, 0.0), 0.0, 0)], 2.0)   # Z = 0: no potential, uniform h = 2


def test_ecs_reduces_to_the_unscaled_operator():
    om = omesh.Mesh(-8.0, 8.0, 4, 2, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)
    op = fem.Operators(om)
    E = (0.01, -0.02, 0.03)
    H0 = op.H1_matrix(E)
    op.set_ecs(0.5, (8.0, 8.0, 8.0))            # the inner box is the whole mesh: nothing scaled
    assert not np.any(op.ecs[2])
    H1 = op.H1_matrix(E)
    assert abs(H1 - H0).max() <= 1e-15 * abs(H0).max()
    op.set_ecs(0.0, (2.0, 2.0, 2.0))            # theta = 0 removes the scaling
    assert op.ecs is None
    assert abs(op.H1_matrix(E) - H0).max() == 0.0


def test_ecs_box_must_not_cut_cells():
    om = omesh.Mesh(*FREE)
    op = fem.Operators(om)
    with pytest.raises(ValueError):
        op.set_ecs(0.3, (5.0, 6.0, 6.0))        # x = +-5 cuts the cells [4, 6] and [-6, -4]


def test_ecs_operator_symmetric_and_decaying():
    """A_theta = A_theta^T (the weak form of a real basis), and every eigenvalue
    of the free kinetic operator 1/2 M_theta^-1 A_theta on the interior has a
    negative imaginary part (all real when theta = 0)."""
    om = omesh.Mesh(-8.0, 8.0, 4, 2, [((0.0, 0.0, 0.0), 0.0, 1)], 2.0)
    op = fem.Operators(om)
    I = np.nonzero(~om.boundary)[0]
    op.set_ecs(0.4, (4.0, 4.0, 4.0))
    At = op.A_theta
    assert abs(At - At.T).max() <= 1e-14 * abs(At).max()
    G = (sp.diags(1.0 / op.ML[I]) @ op.H1_matrix()[I][:, I]).toarray()
    ev = np.linalg.eigvals(G)
    assert ev.imag.max() < -1e-3
    op.set_ecs(0.0, (4.0, 4.0, 4.0))
    ev0 = np.linalg.eigvals((sp.diags(1.0 / op.ML[I]) @ op.H1_matrix()[I][:, I]).toarray())
    assert np.abs(ev0.imag).max() <= 1e-10 * np.abs(ev0).max()


def _free_packet(X, t, sig=1.5, k0=1.0):
    """The exact free-space Gaussian packet (momentum k0 along x) at time t."""
    a = sig ** 2 + 1j * t
    out = np.ones(len(X), dtype=np.complex128)
    for d in range(3):
        k = k0 if d == 0 else 0.0
        x = X[:, d]
        out *= ((sig ** 2 / a) ** 0.5 * np.exp(-(x - k * t) ** 2 / (2 * a) + 1j * k * x - 0.5j * k * k * t)
                * (np.pi * sig ** 2) ** -0.25)
    return out


def test_ecs_absorbs_an_outgoing_packet():
    """A free packet moving out of the inner box |x_d| <= 6: with the scaling
    the inner-box solution at t = 8 stays within 4 % (L2, relative to the
    initial norm) of the exact free packet and the inner norm within 2 %; the
    hard wall (theta = 0) reflects it back (error above 15 %)."""
    om = omesh.Mesh(*FREE)
    op = fem.Operators(om)
    I = np.nonzero(~om.boundary)[0]
    X = om.Xm
    ML = op.ML
    p0 = _free_packet(X, 0.0)
    p0[om.boundary] = 0.0
    T, R = 8.0, 6.0
    pe = _free_packet(X, T)
    inner = np.all(np.abs(X) <= R + 1e-9, axis=1) & ~om.boundary

    def nrm(v, mask):
        return np.sqrt(np.sum(ML[mask] * np.abs(v[mask]) ** 2))

    res = {}
    for theta in (0.0, 0.4):
        op.set_ecs(theta, (R, R, R))
        G = (sp.diags(1.0 / ML[I]) @ op.H1_matrix()[I][:, I]).tocsc()
        pt = np.zeros(om.N, dtype=np.complex128)
        pt[I] = sla.expm_multiply(-1j * T * G, p0[I])
        res[theta] = (nrm(pt - pe, inner) / nrm(p0, ~om.boundary), nrm(pt, inner) ** 2)
    exact_inner = nrm(pe, inner) ** 2
    assert res[0.4][0] < 0.04
    assert abs(res[0.4][1] - exact_inner) < 0.02 * exact_inner
    assert res[0.0][0] > 0.15


def test_ecs_mctdhf_projector_and_ci_norm():
    """With the non-Hermitian one-body operator the projector still removes
    the orbitals' span in <u, v> = u^H M_L v (phi_j^H M_L (G v) = 0), so the
    orbitals stay orthonormal to the scheme's order.  (The scaled operator is
    not dissipative in that inner product, only its spectrum is: the CI norm
    may change either way by a small amount over one step.)"""
    case = (-8.0, 8.0, 4, 2, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    op.set_ecs(0.4, (4.0, 4.0, 4.0))
    solver = mctdhf.MCTDHF(op, 2, 1, 1)
    phi = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, case[4], 2, phase_noise=0.0), op.ML)
    C = inputs.initial_ci(2, 1, 1)
    W, _ = solver.mean_fields(phi)
    g1, g2 = solver.ci.rdm1(C), solver.ci.rdm2(C)
    U = solver.mean_field_operator(g1, g2, W)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(phi.shape) + 1j * rng.standard_normal(phi.shape)
    Gv = solver.G_apply(v, phi, U, (0.0, 0.0, 0.02))
    S = np.conj(phi).T @ (op.ML[:, None] * Gv)
    assert np.abs(S).max() <= 1e-12 * np.abs(Gv).max() * np.sum(op.ML)
    phi1, C1, _info = solver.step(phi, C, (0.0, 0.0, 0.02), 0.01, 10)
    assert abs(np.linalg.norm(C1) - 1.0) < 1e-6
    S1 = np.conj(phi1).T @ (op.ML[:, None] * phi1)
    assert np.abs(S1 - np.eye(2)).max() < 1e-3
