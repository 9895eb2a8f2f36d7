"""GPU parity of afem_poisson_batch against the oracle (Sec. 3.1: Poisson
equation for the mean fields of Eq. mean-field with direct-integral boundary
data).  Judged by backward error in the oracle's assembled matrices, the
surface data element by element, and forward error within kappa * rtol."""
import numpy as np
import pytest

from oracle import fem, mesh as omesh, poisson
from tests._match import coord_permutation

pytestmark = pytest.mark.gpu

CASES = [
    ((-10.0, 10.0, 4, 2, [((0.0, 0.0, 0.0), 1.0, 3)], 2.0), 1),
    ((-8.0, 8.0, 3, 3, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0), 3),
    ((-8.0, 8.0, 3, 4, [((0.3, -0.45, 0.7), 1.0, 2), ((-1.1, 0.2, -0.35), 2.0, 2)], 1.5), 2),
    # 8 orbitals: 64 columns (the water workload's batch), degree 4 (shared tiles above 48 KB)
    ((-8.0, 8.0, 3, 4, [((0.3, -0.45, 0.7), 1.0, 2), ((-1.1, 0.2, -0.35), 2.0, 2)], 1.5), 8),
]


def _orbitals(X, boundary, nuclei, n, seed):
    rng = np.random.default_rng(seed)
    phi = np.zeros((len(X), n), dtype=np.complex128)
    for j in range(n):
        R = np.asarray(nuclei[j % len(nuclei)][0]) + 0.3 * rng.standard_normal(3)
        a = 0.6 + 0.5 * rng.random()
        phase = rng.uniform(-1, 1, 3)
        phi[:, j] = np.exp(-a * np.sum((X - R) ** 2, axis=1)) * np.exp(1j * (X @ phase))
    phi[boundary] = 0
    return phi


@pytest.mark.parametrize("case,n", CASES)
def test_poisson_batch_parity(case, n):
    import torch
    import paper_2301_02387_gb300 as pkg
    lo, hi, nc, p, nuclei, c = case
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    ps = poisson.PoissonSolver(op)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    phi_o = _orbitals(om.Xm, om.boundary, nuclei, n, 17)
    rho, pairs = poisson.pair_densities(op, phi_o)
    Wd = ps.solve(rho, method="cg", rtol=1e-13)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    W = torch.zeros((gm.N, n * n), dtype=torch.float64, device="cuda")
    it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=5000)
    assert rc == 0 and it > 0 and np.all(rel <= 1e-10)
    Wg = np.empty_like(W.cpu().numpy())
    Wg[perm] = W.cpu().numpy()            # back to oracle order
    # surface data element by element (same multipole formula)
    B = om.boundary
    np.testing.assert_allclose(Wg[B], Wd[B], rtol=1e-10, atol=1e-12 * np.abs(Wd[B]).max())
    # backward error in the oracle's assembled matrices
    assert np.all(ps.residual(Wg, rho) < 2e-10)
    # forward error within kappa * rtol (kappa of the Jacobi-scaled Laplacian here < 1e4);
    # the oracle reference is itself a CG solve to rtol 1e-13
    scale = np.abs(Wd).max(axis=0)
    assert np.all(np.abs(Wg - Wd).max(axis=0) <= 1e-6 * scale)
    # warm start from the converged solution: no iteration needed
    it2, rel2, rc2 = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=5000, warm_start=True)
    assert rc2 == 0 and it2 == 0


def test_poisson_batch_zero_density_and_maxit():
    import torch
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(-6.0, 6.0, 3, 2, [((0.0, 0.0, 0.0), 1.0, 2)], 2.0)
    phi = torch.zeros((gm.N, 2), dtype=torch.complex128, device="cuda")
    W = torch.full((gm.N, 4), 7.0, dtype=torch.float64, device="cuda")
    it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=100)
    assert rc == 0 and it == 0
    assert torch.count_nonzero(W).item() == 0
    X, _, _ = gm.tables()
    ph = np.exp(-np.sum(X ** 2, axis=1))
    ph[gm.n_interior:] = 0
    phi = torch.from_numpy(np.stack([ph, 0.5 * ph], axis=1).astype(np.complex128)).cuda()
    it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-12, max_it=3, raise_on_maxit=False)
    assert rc == pkg._capi.AFEM_ECG_MAXIT and it == 3


@pytest.mark.parametrize("case,n", CASES)
@pytest.mark.parametrize("precision_name", ["fp64", "mixed"])
def test_poisson_batch_multigrid_parity(case, n, precision_name):
    """The multigrid-preconditioned solve (AFEM_POISSON_MULTIGRID; FP64 CG, or
    float64 defect correction with float32 corrections) meets the same bars as
    the Jacobi solve: surface data element by element, backward error in the
    oracle's matrices, forward error; in fewer iterations (FP64: a third of the
    Jacobi count at most).  A warm start from the solution needs none."""
    import torch
    import paper_2301_02387_gb300 as pkg
    lo, hi, nc, p, nuclei, c = case
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    ps = poisson.PoissonSolver(op)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    phi_o = _orbitals(om.Xm, om.boundary, nuclei, n, 17)
    rho, pairs = poisson.pair_densities(op, phi_o)
    Wd = ps.solve(rho, method="cg", rtol=1e-13)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    W = torch.zeros((gm.N, n * n), dtype=torch.float64, device="cuda")
    it_jac, _, _ = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=5000)
    pkg.mesh_set_option(gm, pkg.OPT_POISSON_SOLVER, pkg.POISSON_MULTIGRID)
    prec = pkg.PREC_FP64 if precision_name == "fp64" else pkg.PREC_MIXED
    W.zero_()
    it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=5000, precision=prec)
    assert rc == 0 and it > 0 and np.all(rel <= 1e-10)
    if precision_name == "fp64":
        assert it * 3 <= it_jac, (it, it_jac)
    Wg = np.empty_like(W.cpu().numpy())
    Wg[perm] = W.cpu().numpy()
    B = om.boundary
    np.testing.assert_allclose(Wg[B], Wd[B], rtol=1e-10, atol=1e-12 * np.abs(Wd[B]).max())
    assert np.all(ps.residual(Wg, rho) < 2e-10)
    scale = np.abs(Wd).max(axis=0)
    assert np.all(np.abs(Wg - Wd).max(axis=0) <= 1e-6 * scale)
    it2, rel2, rc2 = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=5000, warm_start=True, precision=prec)
    assert rc2 == 0 and it2 == 0


def test_poisson_multigrid_zero_density_and_maxit():
    import torch
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(-6.0, 6.0, 3, 2, [((0.0, 0.0, 0.0), 1.0, 2)], 2.0)
    pkg.mesh_set_option(gm, pkg.OPT_POISSON_SOLVER, pkg.POISSON_MULTIGRID)
    phi = torch.zeros((gm.N, 2), dtype=torch.complex128, device="cuda")
    W = torch.full((gm.N, 4), 7.0, dtype=torch.float64, device="cuda")
    it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=100)
    assert rc == 0 and it == 0
    assert torch.count_nonzero(W).item() == 0
    X, _, _ = gm.tables()
    ph = np.exp(-np.sum(X ** 2, axis=1))
    ph[gm.n_interior:] = 0
    phi = torch.from_numpy(np.stack([ph, 0.5 * ph], axis=1).astype(np.complex128)).cuda()
    it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-14, max_it=1, raise_on_maxit=False)
    assert rc == pkg._capi.AFEM_ECG_MAXIT and it == 1
    with pytest.raises(pkg.AfemError):
        pkg.mesh_set_option(gm, pkg.OPT_POISSON_SOLVER, 7)


def test_poisson_multigrid_on_a_kelly_mesh():
    """The multigrid hierarchy of a Kelly-refined mesh (coarse levels by
    truncating its octree) solves to the oracle's backward-error bar."""
    import torch
    import paper_2301_02387_gb300 as pkg
    case = (-8.0, 8.0, 4, 3, [((0.0, 0.0, 0.7), 1.0, 5), ((0.0, 0.0, -0.7), 1.0, 5)], 2.0)
    gm = pkg.Mesh(*case, kelly=(0.3, 4))
    om = omesh.Mesh(*case, kelly=(0.3, 4))
    op = fem.Operators(om)
    ps = poisson.PoissonSolver(op)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    phi_o = _orbitals(om.Xm, om.boundary, case[4], 2, 5)
    rho, _ = poisson.pair_densities(op, phi_o)
    pkg.mesh_set_option(gm, pkg.OPT_POISSON_SOLVER, pkg.POISSON_MULTIGRID)
    for prec in (pkg.PREC_FP64, pkg.PREC_MIXED):
        phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
        W = torch.zeros((gm.N, 4), dtype=torch.float64, device="cuda")
        it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=5000, precision=prec)
        assert rc == 0 and np.all(rel <= 1e-10)
        Wg = np.empty((om.N, 4))
        Wg[perm] = W.cpu().numpy()
        assert np.all(ps.residual(Wg, rho) < 2e-10)
