"""GPU parity of afem_arnoldi_step (Sec. 3.2, Eq. packed_orb_eom) against the
oracle's Arnoldi on its assembled G operator.  FP64 bar: 1e-10 relative."""
import numpy as np
import pytest

from oracle import fem, krylov, mctdhf, mesh as omesh
from paper_2301_02387_gb300 import inputs
from tests._match import assert_close, coord_permutation

pytestmark = pytest.mark.gpu

CASES = [
    ((-8.0, 8.0, 3, 2, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0), 2, True),
    ((-8.0, 8.0, 3, 3, [((0.3, -0.45, 0.7), 1.0, 2), ((-1.1, 0.2, -0.35), 2.0, 2)], 1.5), 3, True),
    ((-6.0, 6.0, 2, 4, [((0.0, 0.0, 0.0), 1.0, 2)], 2.0), 1, False),
]


def _fields(X, n, seed):
    rng = np.random.default_rng(seed)
    U = np.zeros((n, n, len(X)), dtype=np.complex128)
    for p in range(n):
        for q in range(n):
            c = rng.standard_normal(3)
            U[p, q] = (0.3 + 0.2j * rng.standard_normal()) * np.exp(-0.2 * np.sum((X - c) ** 2, axis=1))
    return U


@pytest.mark.parametrize("case,n,with_U", CASES)
@pytest.mark.parametrize("m", [1, 6, 10])
def test_arnoldi_step_parity(case, n, with_U, m):
    import torch
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    interior = ~om.boundary
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, interior, case[4], n), op.ML)
    U_o = _fields(om.Xm, n, 3) if with_U else np.zeros((n, n, om.N), dtype=np.complex128)
    E = (0.01, -0.02, 0.03)
    sim = mctdhf.MCTDHF.__new__(mctdhf.MCTDHF)
    sim.ops, sim.mesh, sim.n = op, om, n
    sim.interior = interior.astype(np.float64)
    ref, err, H, m_used, brk = krylov.arnoldi_expm(
        lambda v: sim.G_apply(v, phi_o, U_o, E), phi_o, sim.inner, m, 0.02)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    U = torch.from_numpy(np.ascontiguousarray(U_o.transpose(2, 0, 1)[perm])).cuda() if with_U else None
    out, err_g, mu, brk_g = pkg.arnoldi_step(gm, phi, U, m, 0.02, E=E)
    torch.cuda.synchronize()
    assert_close(out.cpu().numpy(), ref[perm], 1e-10, what="Arnoldi step")
    assert mu == m_used and brk_g == brk
    assert abs(err_g - err) <= 1e-6 * abs(err) + 1e-18


def test_arnoldi_eigenvector_breakdown():
    """A discrete eigenvector of M_L^-1 H1~ is a fixed point of G (Q H phi0 = 0)."""
    import scipy.linalg
    import torch
    import paper_2301_02387_gb300 as pkg
    case = (-5.0, 5.0, 2, 2, [((0.0, 0.0, 0.0), 1.0, 1)], 2.0)
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    I = np.nonzero(~om.boundary)[0]
    ev, V = scipy.linalg.eigh(op.H1_matrix().toarray()[np.ix_(I, I)], np.diag(op.ML[I]))
    phi_o = np.zeros((om.N, 1), dtype=np.complex128)
    phi_o[I, 0] = V[:, 0]
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    out, err, mu, brk = pkg.arnoldi_step(gm, phi, None, 8, 0.05)
    assert brk and mu == 1 and err == 0.0
    np.testing.assert_allclose(out.cpu().numpy(), phi_o[perm], atol=1e-10)


@pytest.mark.parametrize("precision_name", ["fp64", "mixed"])
def test_arnoldi_propagate_substeps_parity(precision_name):
    """Error-controlled substepping: same substep count as the oracle; FP64 result
    within 1e-10, the mixed form within 1e-6."""
    import torch
    import paper_2301_02387_gb300 as pkg
    case = (-6.0, 6.0, 2, 3, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    n = 2
    interior = ~om.boundary
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, interior, case[4], n), op.ML)
    U_o = _fields(om.Xm, n, 8)
    E = (0.0, 0.0, 0.02)
    sim = mctdhf.MCTDHF.__new__(mctdhf.MCTDHF)
    sim.ops, sim.mesh, sim.n = op, om, n
    sim.interior = interior.astype(np.float64)
    ref, err, sub = krylov.arnoldi_propagate(lambda v: sim.G_apply(v, phi_o, U_o, E), phi_o, sim.inner, 6, 0.05,
                                             1e-9)
    assert sub > 1
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    U = torch.from_numpy(np.ascontiguousarray(U_o.transpose(2, 0, 1)[perm])).cuda()
    prec = pkg.PREC_FP64 if precision_name == "fp64" else pkg.PREC_MIXED
    out, err_g, sub_g = pkg.arnoldi_propagate(gm, phi, U, 6, 0.05, 1e-9, E=E, precision=prec)
    torch.cuda.synchronize()
    if precision_name == "fp64":
        assert sub_g == sub
        assert_close(out.cpu().numpy(), ref[perm], 1e-10, what="propagation")
    else:
        assert abs(sub_g - sub) <= 1
        assert_close(out.cpu().numpy(), ref[perm], 1e-6, what="propagation")


@pytest.mark.parametrize("precision_name", ["fp64", "mixed"])
def test_arnoldi_adaptive_dimension_parity(precision_name):
    """Sec. 3.2's rule (fixed steps, dimension grown until the estimate passes)
    against the oracle's: the same dimension for every step unless the
    oracle's decisions include a near-tie (margin), FP64 within 1e-10, the
    precision form within 1e-6."""
    import torch
    import paper_2301_02387_gb300 as pkg
    case = (-6.0, 6.0, 2, 3, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    n = 2
    interior = ~om.boundary
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, interior, case[4], n), op.ML)
    U_o = _fields(om.Xm, n, 9)
    E = (0.0, 0.01, 0.02)
    sim = mctdhf.MCTDHF.__new__(mctdhf.MCTDHF)
    sim.ops, sim.mesh, sim.n = op, om, n
    sim.interior = interior.astype(np.float64)
    dt, steps, tol, m_max = 0.05, 4, 1e-10, 16
    ref, err_o, info = krylov.arnoldi_adaptive(lambda v: sim.G_apply(v, phi_o, U_o, E), phi_o, sim.inner, m_max,
                                               dt, tol, substeps=steps)
    assert info["passed"] and min(info["dims"]) >= 4
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    U = torch.from_numpy(np.ascontiguousarray(U_o.transpose(2, 0, 1)[perm])).cuda()
    fp64 = precision_name == "fp64"
    prec = pkg.PREC_FP64 if fp64 else pkg.PREC_MIXED
    out, err, dmax, dsum, unmet = pkg.arnoldi_adaptive(gm, phi, U, m_max, dt, steps, tol, E=E, precision=prec)
    torch.cuda.synchronize()
    assert unmet == 0
    if info["margin"] > (1e-6 if fp64 else 1e-3):
        assert dmax == max(info["dims"]) and dsum == sum(info["dims"])
        assert_close(out.cpu().numpy(), ref[perm], 1e-10 if fp64 else 1e-6, what="adaptive dimension")
    else:
        assert abs(dsum - sum(info["dims"])) <= steps
        assert_close(out.cpu().numpy(), ref[perm], max(1e-6, 4.0 * (err + err_o)), what="near-tie")


def test_arnoldi_adaptive_reports_unmet_threshold():
    """A cap of 3 dimensions cannot meet 1e-12 over the step: every step is
    counted as unmet and uses the cap."""
    import torch
    import paper_2301_02387_gb300 as pkg
    case = (-6.0, 6.0, 2, 3, [((0.0, 0.0, 0.0), 1.0, 2)], 2.0)
    gm = pkg.Mesh(*case)
    X, ml, _ = gm.tables()
    interior = np.arange(gm.N) < gm.n_interior
    phi = torch.from_numpy(inputs.lowdin(inputs.molecular_orbitals(X, interior, case[4], 1), ml)).cuda()
    out, err, dmax, dsum, unmet = pkg.arnoldi_adaptive(gm, phi, None, 3, 0.05, 2, 1e-12)
    assert unmet == 2 and dmax == 3 and dsum == 6
    with pytest.raises(pkg.AfemError):
        pkg.arnoldi_adaptive(gm, phi, None, 17, 0.05, 2, 1e-12)
