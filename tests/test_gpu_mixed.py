"""Precision form (FP32 cell operators, FP64 refinement / Gram-Schmidt / CI)
against the FP64 oracle: the Poisson batch keeps the FP64 backward-error bar,
the Arnoldi step and the MCTDHF step stay within 1e-6 relative."""
import numpy as np
import pytest

from oracle import fem, krylov, mctdhf, mesh as omesh, poisson
from paper_2301_02387_gb300 import inputs
from tests._match import assert_close, coord_permutation

pytestmark = pytest.mark.gpu

CASE = (-8.0, 8.0, 3, 3, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)


@pytest.fixture(scope="module")
def pair():
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(*CASE)
    om = omesh.Mesh(*CASE)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    return gm, om, op, coord_permutation(X, om.Xm)


def test_mixed_poisson_reaches_fp64_backward_error(pair):
    import torch
    import paper_2301_02387_gb300 as pkg
    gm, om, op, perm = pair
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, CASE[4], 3), op.ML)
    ps = poisson.PoissonSolver(op)
    rho, _ = poisson.pair_densities(op, phi_o)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    W = torch.zeros((gm.N, 9), dtype=torch.float64, device="cuda")
    it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=20000, precision=pkg.PREC_MIXED)
    assert rc == 0 and np.all(rel <= 1e-10)
    Wg = np.empty((om.N, 9))
    Wg[perm] = W.cpu().numpy()
    assert np.all(ps.residual(Wg, rho) < 2e-10)


def test_mixed_arnoldi_within_1e6(pair):
    import torch
    import paper_2301_02387_gb300 as pkg
    gm, om, op, perm = pair
    n = 2
    interior = ~om.boundary
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, interior, CASE[4], n), op.ML)
    rng = np.random.default_rng(4)
    U_o = np.zeros((n, n, om.N), dtype=np.complex128)
    for p in range(n):
        for q in range(n):
            U_o[p, q] = (0.3 + 0.1j * rng.standard_normal()) * np.exp(-0.2 * np.sum(om.Xm ** 2, axis=1))
    E = (0.0, 0.0, 0.02)
    sim = mctdhf.MCTDHF.__new__(mctdhf.MCTDHF)
    sim.ops, sim.mesh, sim.n = op, om, n
    sim.interior = interior.astype(np.float64)
    ref, *_ = krylov.arnoldi_expm(lambda v: sim.G_apply(v, phi_o, U_o, E), phi_o, sim.inner, 8, 0.01)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    U = torch.from_numpy(np.ascontiguousarray(U_o.transpose(2, 0, 1)[perm])).cuda()
    out, err, mu, brk = pkg.arnoldi_step(gm, phi, U, 8, 0.01, E=E, precision=pkg.PREC_MIXED)
    torch.cuda.synchronize()
    assert_close(out.cpu().numpy(), ref[perm], 1e-6, what="Arnoldi step")


def test_mixed_mctdhf_steps_within_1e6(pair):
    import torch
    import paper_2301_02387_gb300 as pkg
    gm, om, op, perm = pair
    n, na, nb = 2, 1, 1
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, CASE[4], n), op.ML)
    C_o = inputs.initial_ci(n, na, nb, amp=0.1)
    sim = mctdhf.MCTDHF(op, n, na, nb, poisson_method="cg", poisson_rtol=1e-13)
    solver = pkg.MCTDHF(gm, n, na, nb, 8)
    solver.set_precision(pkg.PREC_MIXED)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    C = torch.from_numpy(C_o.copy()).cuda()
    W = torch.zeros((gm.N, n * n), dtype=torch.float64, device="cuda")
    E = (0.0, 0.0, 0.03)
    for _ in range(3):
        phi_o, C_o, info_o = sim.step(phi_o, C_o, E, 0.01, 8)
        info = solver.step(phi, C, W, E, 0.01, cg_rtol=1e-12)
    torch.cuda.synchronize()
    assert_close(phi.cpu().numpy(), phi_o[perm], 1e-6, what="orbitals")
    assert_close(C.cpu().numpy(), C_o, 1e-6, what="CI vector")
    assert abs(info["energy"] - info_o["energy"]) < 1e-6 * abs(info_o["energy"])
    # orbital norms (sum over orbitals of phi^H M_L phi) agree to 1e-6
    ML = op.ML
    pg = np.empty_like(phi_o)
    pg[perm] = phi.cpu().numpy()
    ng = np.real(np.sum(np.conj(pg) * ML[:, None] * pg, axis=0))
    no = np.real(np.sum(np.conj(phi_o) * ML[:, None] * phi_o, axis=0))
    np.testing.assert_allclose(ng, no, rtol=1e-6)


CASES_N = [
    CASE,
    (-8.0, 8.0, 3, 4, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0),
]


@pytest.mark.parametrize("case", CASES_N)
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("blocks", [1, 2, 0])
def test_arnoldi_orbital_counts_with_mean_field(case, n, blocks):
    """The G cell pass with all n^2 mean fields for odd orbital counts (the
    scalar-lane kernel) and 1 to 4 float4 quads per node (n = 2, 4, 6, 8; 8
    orbitals and 64 fields as in the water workload), degrees 3 and 4, with
    the degree-4 precision form on frozen per-cell blocks staged by bulk copies
    (blocks = 1: one cell per thread block; 2: the pipelined persistent pass
    for n <= 4) and with the mean-field rows gathered in the pass (0): one
    Krylov step of dimension 8, FP64 within 1e-10 of the oracle, the precision
    form within 1e-6."""
    import torch
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(*case)
    pkg.mesh_set_option(gm, pkg.OPT_GCELL_BLOCKS, blocks)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    interior = ~om.boundary
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, interior, case[4], n), op.ML)
    rng = np.random.default_rng(40 + n)
    U_o = np.zeros((n, n, om.N), dtype=np.complex128)
    for p in range(n):
        for q in range(n):
            c = rng.standard_normal(3)
            U_o[p, q] = (0.3 + 0.2j * rng.standard_normal()) * np.exp(-0.2 * np.sum((om.Xm - c) ** 2, axis=1))
    E = (0.01, -0.02, 0.03)
    sim = mctdhf.MCTDHF.__new__(mctdhf.MCTDHF)
    sim.ops, sim.mesh, sim.n = op, om, n
    sim.interior = interior.astype(np.float64)
    ref, *_ = krylov.arnoldi_expm(lambda v: sim.G_apply(v, phi_o, U_o, E), phi_o, sim.inner, 8, 0.01)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    U = torch.from_numpy(np.ascontiguousarray(U_o.transpose(2, 0, 1)[perm])).cuda()
    for prec, bar in ((pkg.PREC_FP64, 1e-10), (pkg.PREC_MIXED, 1e-6)):
        out, err, mu, brk = pkg.arnoldi_step(gm, phi, U, 8, 0.01, E=E, precision=prec)
        torch.cuda.synchronize()
        assert_close(out.cpu().numpy(), ref[perm], bar, what=f"precision {prec}")


@pytest.mark.parametrize("n", [2, 4, 6, 8])
@pytest.mark.parametrize("variant", [0, 2])
def test_mixed_poisson_column_counts(pair, n, variant):
    """The precision form's Poisson batch for 4 and 16 columns (fused p.Ap), 36
    and 64 columns (9 and 16 float4 quads per node: the run-time quad count),
    with the node-per-thread and the column-pair line stiffness pass: FP64
    backward error <= 2e-10 in the oracle's matrices."""
    import torch
    import paper_2301_02387_gb300 as pkg
    gm, om, op, perm = pair
    pkg.mesh_set_option(gm, pkg.OPT_CELL32_VARIANT, variant)
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, CASE[4], n), op.ML)
    ps = poisson.PoissonSolver(op)
    rho, _ = poisson.pair_densities(op, phi_o)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    W = torch.zeros((gm.N, n * n), dtype=torch.float64, device="cuda")
    try:
        it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=20000, precision=pkg.PREC_MIXED)
    finally:
        pkg.mesh_set_option(gm, pkg.OPT_CELL32_VARIANT, 0)
    assert rc == 0 and np.all(rel <= 1e-10)
    Wg = np.empty((om.N, n * n))
    Wg[perm] = W.cpu().numpy()
    assert np.all(ps.residual(Wg, rho) < 2e-10)


def test_mixed_mctdhf_water_shaped_within_1e6():
    """Precision form of the MCTDHF step with 8 orbitals (1 alpha + 1 beta) on
    a small O + 2 H mesh: within 1e-6 of the oracle over 2 steps."""
    import torch
    import paper_2301_02387_gb300 as pkg
    case = (-6.0, 6.0, 2, 3, [((0.0, 0.0, 0.0), 8.0, 1), ((1.4311, 1.1081, 0.0), 1.0, 1),
                              ((-1.4311, 1.1081, 0.0), 1.0, 1)], 2.0)
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    n, na, nb = 8, 1, 1
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, case[4], n), op.ML)
    C_o = inputs.initial_ci(n, na, nb, amp=0.1)
    sim = mctdhf.MCTDHF(op, n, na, nb, poisson_method="cg", poisson_rtol=1e-13)
    solver = pkg.MCTDHF(gm, n, na, nb, 8)
    solver.set_precision(pkg.PREC_MIXED)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    C = torch.from_numpy(C_o.copy()).cuda()
    W = torch.zeros((gm.N, n * n), dtype=torch.float64, device="cuda")
    E = (0.0, 0.01, 0.03)
    for _ in range(2):
        phi_o, C_o, info_o = sim.step(phi_o, C_o, E, 0.02, 8)
        info = solver.step(phi, C, W, E, 0.02, cg_rtol=1e-12)
    torch.cuda.synchronize()
    assert_close(phi.cpu().numpy(), phi_o[perm], 1e-6, what="orbitals")
    assert_close(C.cpu().numpy(), C_o, 1e-6, what="CI vector")
    assert abs(info["energy"] - info_o["energy"]) < 1e-6 * abs(info_o["energy"])
