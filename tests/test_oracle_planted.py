"""Planted mistakes: each test plants one plausible mistake in the oracle
(monkeypatched, on the CPU only) and checks that one of the oracle's pins then
fails.  This is evidence that the pins constrain the parts they are meant to:
a dropped term, a wrong sign or factor, a conjugated or transposed operand,
weights attached to the wrong unknowns."""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint, ci, fem, gll, krylov, mctdhf, mesh, poisson, rows, step_grad
from paper_2301_02387_gb300 import inputs
from tests import test_oracle_adjoint as T_adj
from tests import test_oracle_fem as T_fem
from tests import test_oracle_mctdhf as T_mc
from tests import test_oracle_mesh as T_mesh
from tests import test_oracle_poisson as T_poi
from tests import test_oracle_rows as T_rows
from tests import test_oracle_step_grad as T_sg


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_stiffness_with_one_direction_dropped(monkeypatch):
    orig = fem.cell_matrices

    def planted(p):
        A_hat, m_hat = orig(p)
        _, w = gll.gll_nodes_weights(p)
        W = np.diag(w)
        return A_hat - np.kron(gll.stiffness_1d(p), np.kron(W, W)), m_hat

    monkeypatch.setattr(fem, "cell_matrices", planted)
    _fails(T_fem.test_stiffness_identities, 2)


def test_coulomb_potential_with_the_wrong_sign(monkeypatch):
    orig = fem.Operators.nuclear_potential
    monkeypatch.setattr(fem.Operators, "nuclear_potential", lambda self, X: -orig(self, X))
    _fails(T_fem.test_hydrogen_rayleigh_quotient_h_convergence, 2, 2)


def test_field_term_with_the_wrong_sign(monkeypatch):
    orig = fem.Operators.H1_matrix
    monkeypatch.setattr(fem.Operators, "H1_matrix",
                        lambda self, E=(0.0, 0.0, 0.0): orig(self, tuple(-np.asarray(E, dtype=float))))
    _fails(T_fem.test_dipole_term_sign_and_axis)


def test_hanging_weights_on_the_wrong_masters(monkeypatch):
    orig = mesh.Mesh._build_constraints

    def planted(self):
        orig(self)
        C = self.C
        for r in np.nonzero(self.hanging)[0]:
            a, b = C.indptr[r], C.indptr[r + 1]
            C.data[a:b] = C.data[a:b][::-1].copy()

    monkeypatch.setattr(mesh.Mesh, "_build_constraints", planted)
    _fails(T_mesh.test_constraints_reproduce_q_p_polynomials, 2)


def test_poisson_right_hand_side_without_4_pi(monkeypatch):
    orig = poisson.PoissonSolver.rhs_and_bc

    def planted(self, rho_f):
        b, g = orig(self, rho_f)
        return b / (4.0 * math.pi), g

    monkeypatch.setattr(poisson.PoissonSolver, "rhs_and_bc", planted)
    m = mesh.Mesh(-10.0, 10.0, 4, 3, [((0.0, 0.0, 0.0), 1.0, 3)], 2.0)
    op = fem.Operators(m)
    _fails(T_poi.test_gaussian_charge_potential_and_self_energy, (m, op, poisson.PoissonSolver(op)))


def test_multipole_potential_with_r_to_the_l(monkeypatch):
    def planted(q, Xb, center, lmax=poisson.LMAX):
        r, th, ph = poisson._spherical(Xb, center)
        k = next(iter(q.values())).shape[0]
        g = np.zeros((len(Xb), k))
        for l in range(lmax + 1):
            fac = 4.0 * math.pi / (2 * l + 1) / r ** l
            for mm in range(-l, l + 1):
                g += np.outer(fac * poisson.real_sph_harm(l, mm, th, ph), q[(l, mm)])
        return g

    monkeypatch.setattr(poisson, "multipole_potential", planted)
    _fails(T_poi.test_multipole_matches_direct_sum_off_centre)


def test_two_body_density_without_the_delta_term(monkeypatch):
    orig = ci.CISpace.rdm2

    def planted(self, C):
        G = orig(self, C)
        g1 = self.rdm1(C)
        for q in range(self.n):
            G[:, q, q, :] += g1
        return G

    monkeypatch.setattr(ci.CISpace, "rdm2", planted)
    _fails(T_mc.test_rdm_traces_and_closed_shell_energy)


def test_arnoldi_with_the_inner_product_arguments_swapped(monkeypatch):
    orig = krylov.arnoldi_expm
    monkeypatch.setattr(krylov, "arnoldi_expm",
                        lambda G, phi, inner, m, dt, **kw: orig(G, phi, lambda u, v: inner(v, u), m, dt, **kw))
    _fails(T_mc.test_arnoldi_step_is_the_galerkin_projection_on_the_krylov_space, 6)


def test_arnoldi_basis_with_the_inner_product_arguments_swapped(monkeypatch):
    orig = krylov.arnoldi_basis
    monkeypatch.setattr(krylov, "arnoldi_basis",
                        lambda G, phi, inner, m, **kw: orig(G, phi, lambda u, v: inner(v, u), m, **kw))
    _fails(T_mc.test_arnoldi_basis_is_orthonormal_with_projected_hessenberg)


def test_adjoint_recursion_with_the_propagator_not_its_adjoint(monkeypatch):
    om = mesh.Mesh(*T_adj.CASE)
    op = fem.Operators(om)
    td = adjoint.TDSE(op, e_dir=(0.0, 0.0, 1.0))
    phi = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, T_adj.CASE[4], 1), op.ML)[:, 0]
    monkeypatch.setattr(adjoint.TDSE, "adjoint_of", lambda self, A: A)
    _fails(T_adj.test_adjoint_state_is_gradient_wrt_initial_state, (td, td.restrict(phi)))


def test_row_oracle_without_the_constraint_transpose(monkeypatch):
    orig = rows.RowOperators.__init__

    def planted(self, m):
        orig(self, m)
        CT = self.CT.tocoo()
        keep = CT.col == m.master_pts[CT.row]
        self.CT = type(self.CT)((CT.data[keep], (CT.row[keep], CT.col[keep])), shape=CT.shape)

    monkeypatch.setattr(rows.RowOperators, "__init__", planted)
    _fails(T_rows.test_rows_equal_assembled_operators, T_rows.CASES[0])


def test_dense_step_with_the_two_electron_term_doubled(monkeypatch):
    orig = step_grad.DenseMCTDHF.__init__

    def planted(self, sim, e_dir=(0.0, 0.0, 1.0)):
        orig(self, sim, e_dir)
        self.E2 = 2.0 * self.E2

    om = mesh.Mesh(*T_sg.CASE)
    op = fem.Operators(om)
    sim = mctdhf.MCTDHF(op, 2, 1, 1)
    monkeypatch.setattr(step_grad.DenseMCTDHF, "__init__", planted)
    dm = step_grad.DenseMCTDHF(sim, e_dir=(0.3, -0.4, 0.866))
    phi = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, T_sg.CASE[4], 2), op.ML)
    C = inputs.initial_ci(2, 1, 1, amp=0.1)
    with torch.no_grad():
        _fails(T_sg.test_dense_step_equals_oracle_step, (sim, dm, phi, C))


def test_two_electron_integrals_with_r_and_s_swapped(monkeypatch):
    orig = mctdhf.MCTDHF.integrals

    def planted(self, phi, W, E):
        h, eri = orig(self, phi, W, E)
        return h, eri.transpose(0, 1, 3, 2)

    monkeypatch.setattr(mctdhf.MCTDHF, "integrals", planted)
    _fails(T_mc.test_integrals_symmetries_with_complex_orbitals)


def test_mean_field_operator_with_gamma_not_inverted(monkeypatch):
    monkeypatch.setattr(mctdhf.MCTDHF, "mean_field_operator",
                        lambda self, g1, g2, W: np.einsum("pqrs,rsk->pqk", np.einsum("po,oqrs->pqrs", g1, g2), W))
    m = mesh.Mesh(*T_mc.TINY)
    _fails(T_mc.test_two_electron_closed_shell_is_tdhf, (m, fem.Operators(m)))


def test_orbital_operator_without_the_projector(monkeypatch):
    orig = mctdhf.MCTDHF.G_apply
    monkeypatch.setattr(mctdhf.MCTDHF, "G_apply",
                        lambda self, v, phi, U, E: orig(self, v, np.zeros_like(phi), U, E))
    m = mesh.Mesh(*T_mc.TINY)
    _fails(T_mc.test_eigenvector_is_stationary, (m, fem.Operators(m)))


def test_ci_hamiltonian_without_the_delta_term(monkeypatch):
    orig = ci.CISpace.hamiltonian

    def planted(self, h, eri):
        H = orig(self, h, eri)
        for p in range(self.n):
            for q in range(self.n):
                for s in range(self.n):
                    H = H + 0.5 * eri[p, q, q, s] * self.E[p][s].toarray()
        return H

    monkeypatch.setattr(ci.CISpace, "hamiltonian", planted)
    _fails(T_mc.test_ci_two_electron_first_quantised)


def test_pair_densities_conjugating_the_wrong_factor(monkeypatch):
    orig = poisson.pair_densities

    def planted(ops, phi):
        rho, pairs = orig(ops, phi)
        for j, (_r, _s, part) in enumerate(pairs):
            if part == 1:
                rho[:, j] = -rho[:, j]
        return rho, pairs

    monkeypatch.setattr(poisson, "pair_densities", planted)
    _fails(T_mc.test_integrals_symmetries_with_complex_orbitals)


def test_multipole_moments_without_the_quadrature_weights(monkeypatch):
    orig = poisson.multipole_moments
    monkeypatch.setattr(poisson, "multipole_moments",
                        lambda X, w, rho, c, lmax=poisson.LMAX: orig(X, np.ones_like(w), rho, c, lmax))
    _fails(T_poi.test_multipole_matches_direct_sum_off_centre)


def test_nuclear_force_with_the_wrong_sign(monkeypatch):
    orig = fem.Operators.nuclear_force
    monkeypatch.setattr(fem.Operators, "nuclear_force", lambda self, X: -orig(self, X))
    _fails(T_adj.test_nuclear_force_is_minus_grad_potential)
