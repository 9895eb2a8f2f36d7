"""Pins for the oracle's Arnoldi propagator (Sec. 3.2), CI algebra (Sec. 2) and
MCTDHF step (Eqs. ci_eom, orb_eom, packed_orb_eom)."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import ci, fem, krylov, mctdhf, mesh
from paper_2301_02387_gb300 import inputs

TINY = (-4.0, 4.0, 2, 2, [((0.0, 0.0, 0.35), 1.0, 1), ((0.0, 0.0, -0.35), 1.0, 1)], 2.0)


@pytest.fixture(scope="module")
def tiny():
    m = mesh.Mesh(*TINY)
    return m, fem.Operators(m)


# ------------------------------------------------------------------ Arnoldi
def test_arnoldi_full_dimension_is_exact_dense_expm():
    rng = np.random.default_rng(0)
    n = 30
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    w = rng.random(n) + 0.5
    phi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    inner = lambda u, v: np.sum(np.conj(u) * w * v)
    out, err, H, m_used, brk = krylov.arnoldi_expm(lambda v: G @ v, phi, inner, n, 0.05)
    ref = scipy.linalg.expm(-1j * 0.05 * G) @ phi
    assert np.linalg.norm(out - ref) < 1e-11 * np.linalg.norm(ref)


def _krylov_case(seed=5, n=40):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    G /= np.linalg.norm(G, 2)
    w = rng.random(n) + 0.5
    phi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return G, w, phi, (lambda u, v: np.sum(np.conj(u) * w * v))


@pytest.mark.parametrize("m", [6, 8])
def test_arnoldi_step_is_the_galerkin_projection_on_the_krylov_space(m):
    """Below full dimension the step equals its definition, formed without
    Gram-Schmidt: Q exp(-i dt Q^H W G Q) Q^H W phi with Q a W-orthonormal basis
    of span{phi, G phi, .., G^(m-1) phi} (QR of the weighted Krylov matrix).  At
    full dimension any coefficients satisfy the Arnoldi relation, so only this
    pins the orthogonalisation itself."""
    G, w, phi, inner = _krylov_case()
    dt = 0.7
    out, *_ = krylov.arnoldi_expm(lambda v: G @ v, phi, inner, m, dt)
    K = np.stack([np.linalg.matrix_power(G, k) @ phi for k in range(m)], axis=1)
    sw = np.sqrt(w)
    Qt, _ = np.linalg.qr(sw[:, None] * K)
    Q = Qt / sw[:, None]
    Hq = Q.conj().T @ (w[:, None] * (G @ Q))
    ref = Q @ (scipy.linalg.expm(-1j * dt * Hq) @ (Q.conj().T @ (w * phi)))
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)


def test_arnoldi_basis_is_orthonormal_with_projected_hessenberg():
    """The basis of the substep propagation: <v_i, v_j> = delta_ij and
    h_ij = <v_i, G v_j> (the Galerkin projection), v_1 = phi / beta."""
    G, w, phi, inner = _krylov_case(seed=6)
    m = 8
    beta, V, H, mu, brk, hlast = krylov.arnoldi_basis(lambda v: G @ v, phi, inner, m)
    assert mu == m and not brk
    assert abs(beta - math.sqrt(inner(phi, phi).real)) < 1e-14 * beta
    np.testing.assert_allclose(V[0], phi / beta, rtol=0, atol=1e-15)
    gram = np.array([[inner(V[i], V[j]) for j in range(m + 1)] for i in range(m + 1)])
    assert np.abs(gram - np.eye(m + 1)).max() < 1e-13
    for j in range(m):
        for i in range(j + 2):
            assert abs(H[i, j] - inner(V[i], G @ V[j])) < 1e-13


def test_arnoldi_estimate_bounds_truncation_error():
    rng = np.random.default_rng(1)
    n = 60
    A = rng.standard_normal((n, n))
    G = (A + A.T) + 0.3 * rng.standard_normal((n, n))
    phi = rng.standard_normal(n) + 0j
    inner = lambda u, v: np.vdot(u, v)
    ref = scipy.linalg.expm(-1j * 0.02 * G) @ phi
    errs = []
    for m in (4, 6, 8):
        out, est, *_ = krylov.arnoldi_expm(lambda v: G @ v, phi, inner, m, 0.02)
        true = np.linalg.norm(out - ref)
        errs.append(true)
        assert true < 5.0 * est + 1e-13
    assert errs[0] > errs[1] > errs[2]


def test_arnoldi_happy_breakdown_on_eigenvector():
    G = np.diag([1.0, 2.0, 3.0]).astype(complex)
    phi = np.array([0.0, 1.0, 0.0], dtype=complex)
    out, err, H, m_used, brk = krylov.arnoldi_expm(lambda v: G @ v, phi, lambda u, v: np.vdot(u, v), 5, 0.1)
    assert brk and m_used == 1 and err == 0.0
    np.testing.assert_allclose(out, np.exp(-0.2j) * phi, atol=1e-15)


# ----------------------------------------------------------------------- CI
def test_ci_two_electron_first_quantised():
    """For 1 alpha + 1 beta electron, H_CI acting on C_pq equals
    h C + C h^T + sum_rs (pr|qs) C_rs (the two-particle Schroedinger operator)."""
    n = 3
    rng = np.random.default_rng(2)
    h = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    h = h + h.conj().T
    eri = rng.standard_normal((n, n, n, n)) + 1j * rng.standard_normal((n, n, n, n))
    eri = eri + eri.transpose(2, 3, 0, 1)                 # (pq|rs) = (rs|pq)
    eri = eri + eri.transpose(1, 0, 3, 2).conj()          # (pq|rs) = (qp|sr)^*
    space = ci.CISpace(n, 1, 1)
    H = space.hamiltonian(h, eri)
    Cm = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    # alpha string of orbital p has bit-mask 1 << p -> index p; likewise beta
    ref = h @ Cm + Cm @ h.T + np.einsum("prqs,rs->pq", eri, Cm)
    out = (H @ Cm.ravel()).reshape(n, n)
    np.testing.assert_allclose(out, ref, atol=1e-12)
    np.testing.assert_allclose(H, H.conj().T, atol=1e-12)


def test_rdm_traces_and_closed_shell_energy():
    n, na, nb = 4, 2, 2
    space = ci.CISpace(n, na, nb)
    C = inputs.initial_ci(n, na, nb, seed=5, amp=0.2)
    g1 = space.rdm1(C)
    g2 = space.rdm2(C)
    Ne = na + nb
    assert abs(np.trace(g1) - Ne) < 1e-12
    assert abs(np.einsum("pprr->", g2) - Ne * (Ne - 1)) < 1e-11
    np.testing.assert_allclose(g1, g1.conj().T, atol=1e-14)
    np.testing.assert_allclose(g2, g2.transpose(2, 3, 0, 1), atol=1e-14)
    ev = np.linalg.eigvalsh(g1)
    assert ev.min() > -1e-12 and ev.max() < 2 + 1e-12
    # closed-shell determinant: E = 2 sum_i h_ii + sum_ij [2 (ii|jj) - (ij|ji)]
    rng = np.random.default_rng(3)
    h = rng.standard_normal((n, n))
    h = h + h.T
    eri = rng.standard_normal((n, n, n, n))
    eri = eri + eri.transpose(1, 0, 2, 3)
    eri = eri + eri.transpose(0, 1, 3, 2)
    eri = eri + eri.transpose(2, 3, 0, 1)
    H = space.hamiltonian(h, eri)
    occ = range(na)
    E = 2 * sum(h[i, i] for i in occ) + sum(2 * eri[i, i, j, j] - eri[i, j, j, i] for i in occ for j in occ)
    assert abs(H[0, 0] - E) < 1e-12


def test_integrals_symmetries_with_complex_orbitals():
    """With orbitals of large complex phase: (pq|rs) = conj((qp|sr)) and
    h_pq = conj(h_qp) exactly, and the Coulomb pair symmetry (pq|rs) = (rs|pq)
    up to the truncation of the multipole surface data (the discrete solve is
    otherwise symmetric); an (r, s) index slip breaks the latter by O(1)."""
    case = (-6.0, 6.0, 2, 2, [((0.0, 0.0, 0.7), 1.0, 1), ((0.0, 0.0, -0.7), 1.0, 1)], 2.0)
    m = mesh.Mesh(*case)
    op = fem.Operators(m)
    n = 3
    phi = np.zeros((m.N, n), dtype=complex)
    ks = [(0.8, 0.0, 0.3), (-0.5, 0.9, 0.0), (0.0, -0.7, 1.1)]
    for j in range(n):
        c = np.array([0.3 * j, -0.2, 0.1 * j])
        phi[:, j] = np.exp(-0.8 * np.sum((m.Xm - c) ** 2, axis=1)) * np.exp(1j * m.Xm @ np.array(ks[j]))
    phi[m.boundary] = 0
    phi = inputs.lowdin(phi, op.ML)
    sim = mctdhf.MCTDHF(op, n, 2, 1)
    W, _ = sim.mean_fields(phi)
    h, eri = sim.integrals(phi, W, (0.0, 0.01, 0.02))
    scale = np.abs(eri).max()
    assert np.abs(eri.imag).max() > 0.1 * scale
    np.testing.assert_allclose(eri, eri.transpose(1, 0, 3, 2).conj(), rtol=0, atol=1e-14 * scale)
    np.testing.assert_allclose(h, h.conj().T, rtol=0, atol=1e-13 * np.abs(h).max())
    assert np.abs(eri - eri.transpose(2, 3, 0, 1)).max() < 1e-3 * scale


# ------------------------------------------------------------------- MCTDHF
def _one_electron_setup(tiny):
    m, op = tiny
    interior = ~m.boundary
    phi = inputs.gaussian_orbital(m.Xm, interior, alpha=1.0)[:, None]
    phi = inputs.lowdin(phi, op.ML)
    return m, op, phi


def test_one_electron_step_reduces_to_tdse(tiny):
    """One orbital, one electron: Psi = C phi follows exp(-i H t) Psi0 with a
    first-order error: halving dt halves the deviation."""
    m, op, phi0 = _one_electron_setup(tiny)
    I = np.nonzero(~m.boundary)[0]
    Hd = op.H1_matrix((0.0, 0.0, 0.05)).toarray()[np.ix_(I, I)] / op.ML[I][:, None]
    T = 0.4
    ref = scipy.linalg.expm(-1j * T * Hd) @ phi0[I, 0]
    sim = mctdhf.MCTDHF(op, 1, 1, 0)
    devs = []
    for dt in (0.1, 0.05):
        phi, C = phi0.copy(), np.array([1.0 + 0j])
        for _ in range(int(round(T / dt))):
            phi, C, info = sim.step(phi, C, (0.0, 0.0, 0.05), dt, 12)
        devs.append(np.linalg.norm(C[0] * phi[I, 0] - ref))
    assert 0.4 < devs[1] / devs[0] < 0.6      # first order in dt
    assert devs[1] < 0.05


def test_eigenvector_is_stationary(tiny):
    """Q H1 phi0 = 0 for an eigenvector: the orbital does not move (breakdown) and
    C picks up exp(-i eps dt)."""
    m, op, _ = _one_electron_setup(tiny)
    I = np.nonzero(~m.boundary)[0]
    Hd = op.H1_matrix().toarray()[np.ix_(I, I)]
    ev, V = scipy.linalg.eigh(Hd, np.diag(op.ML[I]))
    phi = np.zeros((m.N, 1), dtype=complex)
    phi[I, 0] = V[:, 0]
    sim = mctdhf.MCTDHF(op, 1, 1, 0)
    phi1, C1, info = sim.step(phi, np.array([1.0 + 0j]), (0.0, 0.0, 0.0), 0.05, 8)
    assert info["breakdown"] and info["m_used"] == 1
    np.testing.assert_allclose(phi1, phi, atol=1e-11)
    assert abs(C1[0] - np.exp(-0.05j * ev[0])) < 1e-12


def test_two_electron_closed_shell_is_tdhf(tiny):
    """n = 1, one alpha + one beta: gamma = 2, Gamma = 2, so U = W_11 (time-dependent
    Hartree-Fock); field-free energy drift shrinks with dt."""
    m, op, phi0 = _one_electron_setup(tiny)
    sim = mctdhf.MCTDHF(op, 1, 1, 1)
    C0 = np.array([1.0 + 0j])
    g1, g2 = sim.ci.rdm1(C0), sim.ci.rdm2(C0)
    assert abs(g1[0, 0] - 2) < 1e-15 and abs(g2[0, 0, 0, 0] - 2) < 1e-15
    W, _ = sim.mean_fields(phi0)
    U = sim.mean_field_operator(g1, g2, W)
    np.testing.assert_allclose(U[0, 0], W[0, 0], atol=1e-15)
    E0 = sim.energy(phi0, C0)
    drifts = []
    for dt in (0.04, 0.02):
        phi, C = phi0.copy(), C0.copy()
        for _ in range(int(round(0.16 / dt))):
            phi, C, _ = sim.step(phi, C, (0.0, 0.0, 0.0), dt, 10)
        drifts.append(abs(sim.energy(phi, C) - E0))
    assert drifts[1] < 0.7 * drifts[0]


def test_h2_like_two_orbital_invariants(tiny):
    m, op = tiny
    interior = ~m.boundary
    phi = inputs.lowdin(inputs.molecular_orbitals(m.Xm, interior, TINY[4], 2), op.ML)
    C0 = inputs.initial_ci(2, 1, 1, amp=0.1)
    sim = mctdhf.MCTDHF(op, 2, 1, 1)
    E = (0.0, 0.0, 0.02)
    drift = []
    for dt in (0.02, 0.01):
        p, C = phi.copy(), C0.copy()
        for _ in range(int(round(0.06 / dt))):
            p, C, info = sim.step(p, C, E, dt, 10)
            assert abs(np.linalg.norm(C) - 1.0) < 1e-13
            assert abs(np.trace(info["gamma"]) - 2.0) < 1e-12
            assert info["arnoldi_err"] < 1e-10
        S = np.conj(p).T @ (op.ML[:, None] * p)
        drift.append(np.abs(S - np.eye(2)).max())
    # the frozen-operator step is first order: orthonormality drift ~ dt
    assert 0.4 < drift[1] / drift[0] < 0.6 and drift[0] < 2e-3


def test_arnoldi_propagate_meets_tolerance_on_stiff_operator():
    """A stiff Hermitian operator (eigenvalues up to 400) over dt = 0.05 with m = 6:
    one Krylov step is far off, substeps controlled by the estimate land within
    a small multiple of tol * substeps of the dense exponential."""
    rng = np.random.default_rng(5)
    n = 80
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-1, 1, n - 10), rng.uniform(200, 400, 10)])
    G = (Q * lam) @ Q.T
    phi = rng.standard_normal(n) + 0j
    inner = lambda u, v: np.vdot(u, v)
    ref = scipy.linalg.expm(-1j * 0.05 * G) @ phi
    one, est1, *_ = krylov.arnoldi_expm(lambda v: G @ v, phi, inner, 6, 0.05)
    assert np.linalg.norm(one - ref) > 1e-3 * np.linalg.norm(ref)
    out, est, sub = krylov.arnoldi_propagate(lambda v: G @ v, phi, inner, 6, 0.05, 1e-10)
    assert sub > 1
    assert np.linalg.norm(out - ref) < 50 * 1e-10 * sub * np.linalg.norm(phi)


def _stiff_case(seed=5, n=80):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-1, 1, n - 10), rng.uniform(200, 400, 10)])
    G = (Q * lam) @ Q.T
    phi = rng.standard_normal(n) + 0j
    return G, phi, (lambda u, v: np.vdot(u, v))


def test_arnoldi_adaptive_dimension_meets_tolerance_and_is_minimal():
    """Sec. 3.2's rule (fixed step, dimension grown until the estimate passes):
    on the stiff operator, 8 equal steps over dt = 0.05 land within a small
    multiple of tol * steps of the dense exponential; every step's dimension
    is the smallest whose estimate passes (the fixed-dimension step one below
    it fails the threshold, the one at it passes)."""
    G, phi, inner = _stiff_case()
    dt, tol, S = 0.05, 1e-10, 8
    ref = scipy.linalg.expm(-1j * dt * G) @ phi
    out, est, info = krylov.arnoldi_adaptive(lambda v: G @ v, phi, inner, 16, dt, tol, substeps=S)
    assert info["passed"] and len(info["dims"]) == S and est <= S * tol * np.linalg.norm(phi) * 1.0001
    assert np.linalg.norm(out - ref) < 50 * tol * S * np.linalg.norm(phi)
    # minimality, step by step from the oracle's own intermediate vectors
    cur = phi
    for d in info["dims"]:
        beta = np.sqrt(inner(cur, cur).real)
        nxt, e_at, *_ = krylov.arnoldi_expm(lambda v: G @ v, cur, inner, d, dt / S)
        assert e_at <= tol * beta
        if d > 1:
            _, e_below, *_ = krylov.arnoldi_expm(lambda v: G @ v, cur, inner, d - 1, dt / S)
            assert e_below > tol * beta
        cur = nxt
    assert np.linalg.norm(cur - out) < 1e-12 * np.linalg.norm(out)


def test_arnoldi_adaptive_reports_an_unmet_threshold_and_breakdown():
    """A dimension cap too small for the step is reported (passed False, the
    cap used); an eigenvector stops at dimension 1 with the exact phase."""
    G, phi, inner = _stiff_case(seed=6)
    out, est, info = krylov.arnoldi_adaptive(lambda v: G @ v, phi, inner, 4, 0.05, 1e-10, substeps=1)
    assert not info["passed"] and info["dims"] == [4] and est > 1e-10 * np.linalg.norm(phi)
    D = np.diag([1.0, 2.0, 3.0]).astype(complex)
    e = np.array([0.0, 1.0, 0.0], dtype=complex)
    out, est, info = krylov.arnoldi_adaptive(lambda v: D @ v, e, lambda u, v: np.vdot(u, v), 6, 0.1, 1e-12,
                                             substeps=2)
    assert info["dims"] == [1, 1] and est == 0.0
    np.testing.assert_allclose(out, np.exp(-0.2j) * e, atol=1e-15)


# ------------------------------------------------------------ imaginary time
def test_imaginary_time_one_electron_reaches_the_lowest_eigenvalue(tiny):
    """One electron (no mean field): imaginary-time steps converge to the lowest
    generalized eigenvalue of (H1~, M_L) on the interior (scipy eigh); the
    energy decreases monotonically."""
    m, op, phi0 = _one_electron_setup(tiny)
    I = np.nonzero(~m.boundary)[0]
    lam = scipy.linalg.eigh(op.H1_matrix().toarray()[np.ix_(I, I)], np.diag(op.ML[I]), eigvals_only=True)[0]
    sim = mctdhf.MCTDHF(op, 1, 1, 0)
    phi, C = phi0.copy(), np.array([1.0 + 0j])
    energies = []
    for _ in range(40):
        phi, C, info = sim.step_imaginary(phi, C, 1.0, 12, krylov_tol=1e-12)
        energies.append(info["energy"])
    assert all(b <= a + 1e-13 for a, b in zip(energies, energies[1:]))
    assert abs(sim.energy(phi, C) - lam) < 1e-9 * abs(lam)
    assert abs(np.sum(op.ML * np.abs(phi[:, 0]) ** 2) - 1.0) < 1e-13


def _scf_closed_shell(sim, op, phi, iters=200):
    """Closed-shell Hartree-Fock of two electrons in one orbital by the
    Roothaan fixed point, an independent route to the stationary state:
    phi <- lowest generalized eigenvector of H1~ + F[V] on the interior, with
    the Hartree potential V damped (V <- (V + W(|phi|^2)) / 2, which removes
    the fixed point's two-cycle); energy 2 h + (00|00)."""
    m = op.mesh
    I = np.nonzero(~m.boundary)[0]
    H1 = op.H1_matrix()
    V = sim.mean_fields(phi)[0][0, 0].real
    for _ in range(iters):
        F = (H1 + op.pointwise(op.C @ V)).toarray()[np.ix_(I, I)]
        ev, X = scipy.linalg.eigh(F, np.diag(op.ML[I]))
        phi = np.zeros((m.N, 1), dtype=np.complex128)
        phi[I, 0] = X[:, 0]
        Wn = sim.mean_fields(phi)[0][0, 0].real
        if np.abs(Wn - V).max() < 1e-13:
            break
        V = 0.5 * (V + Wn)
    h, eri = sim.integrals(phi, sim.mean_fields(phi)[0], (0.0, 0.0, 0.0))
    return phi, (2.0 * h[0, 0] + eri[0, 0, 0, 0]).real


def test_imaginary_time_closed_shell_reaches_hartree_fock(tiny):
    """Two electrons in one orbital: imaginary time converges to the
    closed-shell Hartree-Fock state that the Roothaan fixed point gives."""
    m, op, phi0 = _one_electron_setup(tiny)
    sim = mctdhf.MCTDHF(op, 1, 1, 1)
    _, e_hf = _scf_closed_shell(sim, op, phi0)
    phi, C = phi0.copy(), np.array([1.0 + 0j])
    energies = []
    for _ in range(80):
        phi, C, info = sim.step_imaginary(phi, C, 0.5, 12, krylov_tol=1e-12)
        energies.append(info["energy"])
    # monotone up to the second-order terms of the frozen-operator step near convergence
    assert all(b <= a + 1e-9 * abs(a) for a, b in zip(energies, energies[1:]))
    assert abs(sim.energy(phi, C) - e_hf) < 1e-8 * abs(e_hf)


def test_imaginary_time_two_orbitals_lower_than_hartree_fock(tiny):
    """Two orbitals, one alpha + one beta electron: the energy decreases
    monotonically, ends below the closed-shell Hartree-Fock energy (the
    variational space contains it) and the orbitals stay orthonormal."""
    m, op = tiny
    interior = ~m.boundary
    phi = inputs.lowdin(inputs.molecular_orbitals(m.Xm, interior, TINY[4], 2, phase_noise=0.0), op.ML)
    C = inputs.initial_ci(2, 1, 1, amp=0.1)
    sim = mctdhf.MCTDHF(op, 2, 1, 1)
    m1, op1, phi1 = _one_electron_setup(tiny)
    _, e_hf = _scf_closed_shell(mctdhf.MCTDHF(op, 1, 1, 1), op, phi1)
    energies = []
    for _ in range(30):
        phi, C, info = sim.step_imaginary(phi, C, 0.5, 12, krylov_tol=1e-12)
        energies.append(info["energy"])
    assert all(b <= a + 1e-9 * abs(a) for a, b in zip(energies, energies[1:]))
    assert sim.energy(phi, C) < e_hf
    S = np.conj(phi).T @ (op.ML[:, None] * phi)
    assert np.abs(S - np.eye(2)).max() < 1e-13


# ------------------------------------------------------------------- dipole
def _dipole_state(case, n, na, nb):
    m = mesh.Mesh(*case)
    op = fem.Operators(m)
    interior = ~m.boundary
    phi = inputs.lowdin(inputs.molecular_orbitals(m.Xm, interior, case[4], n, phase_noise=0.0), op.ML)
    C = inputs.initial_ci(n, na, nb)
    return m, op, phi, C


def test_dipole_is_translation_covariant():
    """Moving the whole system (box, nuclei, orbitals) by a = (t, t, t) changes
    <sum r_i> by N_e a (N_e = tr gamma), whatever the orbitals and CI vector."""
    t = 2.0
    nuclei = [((0.3, 0.1, 0.35), 1.0, 1), ((-0.2, 0.0, -0.35), 1.0, 1)]
    base = (-4.0, 4.0, 2, 2, nuclei, 2.0)
    moved = (-4.0 + t, 4.0 + t, 2, 2, [(tuple(np.asarray(R) + t), Z, L) for (R, Z, L) in nuclei], 2.0)
    out = []
    for case in (base, moved):
        m, op, phi, C = _dipole_state(case, 2, 1, 1)
        sim = mctdhf.MCTDHF(op, 2, 1, 1)
        out.append((sim.dipole(phi, C), np.real(np.trace(sim.ci.rdm1(C)))))
    (d0, ne0), (d1, ne1) = out
    assert abs(ne0 - 2.0) < 1e-12 and abs(ne1 - 2.0) < 1e-12
    np.testing.assert_allclose(d1 - d0, ne0 * t * np.ones(3), rtol=0, atol=1e-10)


def test_dipole_is_the_field_derivative_of_the_energy(tiny):
    """Length gauge: H1~(E) = H1~(0) + sum_d E_d F[x_d] is linear in E, so the
    central difference of the electronic energy in E_d equals <sum r_i>_d."""
    m, op = tiny
    interior = ~m.boundary
    phi = inputs.lowdin(inputs.molecular_orbitals(m.Xm, interior, TINY[4], 2), op.ML)
    C = inputs.initial_ci(2, 1, 1)
    sim = mctdhf.MCTDHF(op, 2, 1, 1)
    d = sim.dipole(phi, C)
    eps = 1e-3
    for k in range(3):
        Ep = np.zeros(3)
        Ep[k] = eps
        fd = (sim.energy(phi, C, Ep) - sim.energy(phi, C, -Ep)) / (2 * eps)
        assert abs(fd - d[k]) <= 1e-9 * max(1.0, abs(d[k]))


def test_triangular_pulse_vector_potential_is_minus_the_field_integral():
    """A(t) of the paper's 400 nm 2-cycle triangular pulse: dA/dt = -E by
    central differences, A = 0 before and after the pulse (no DC term)."""
    I, lam = 8e14, 400.0
    T = 4 * math.pi / (45.5634 / lam)
    for t in np.linspace(0.01 * T, 0.99 * T, 37):
        h = 1e-5
        dA = (inputs.triangular_vector_potential(t + h, I, lam)[0]
              - inputs.triangular_vector_potential(t - h, I, lam)[0]) / (2 * h)
        assert abs(dA + inputs.triangular_pulse(t, I, lam)[0]) < 1e-7
    assert inputs.triangular_vector_potential(-1.0, I, lam) == (0.0, 0.0, 0.0)
    assert abs(inputs.triangular_vector_potential(T * (1 - 1e-12), I, lam)[0]) < 1e-9
