"""GPU parity of afem_mctdhf_step against the oracle's MCTDHF step (Sec. 2,
Sec. 3.2; Eqs. ci_eom, orb_eom, packed_orb_eom).  The GPU Poisson batch runs
to rtol 1e-14 so that its forward error (kappa * rtol) stays far below the
1e-10 bar on orbitals, CI vector, energy and dipole; the oracle solves directly."""
import numpy as np
import pytest

from oracle import fem, mctdhf, mesh as omesh, poisson
from paper_2301_02387_gb300 import inputs
from tests._match import coord_permutation

pytestmark = pytest.mark.gpu

WATER_SMALL = (-6.0, 6.0, 2, 3, [((0.0, 0.0, 0.0), 8.0, 1), ((1.4311, 1.1081, 0.0), 1.0, 1),
                                  ((-1.4311, 1.1081, 0.0), 1.0, 1)], 2.0)

CASES = [
    # (mesh, n_orb, n_alpha, n_beta)
    ((-6.0, 6.0, 3, 2, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0), 2, 1, 1),
    ((-6.0, 6.0, 2, 3, [((0.0, 0.0, 0.0), 3.0, 2), ((1.2, 0.9, 0.0), 1.0, 1)], 2.0), 3, 2, 1),
    # water-shaped: O + 2 H, 8 orbitals (64 mean fields, 64 Poisson columns), 1 alpha + 1 beta
    (WATER_SMALL, 8, 1, 1),
]


@pytest.mark.parametrize("case,n,na,nb", CASES)
def test_mctdhf_steps_parity(case, n, na, nb):
    import torch
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    interior = ~om.boundary
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, interior, case[4], n), op.ML)
    C_o = inputs.initial_ci(n, na, nb, amp=0.1)
    sim = mctdhf.MCTDHF(op, n, na, nb)
    solver = pkg.MCTDHF(gm, n, na, nb, 8)
    assert solver.ci_dim == len(C_o)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    C = torch.from_numpy(C_o.copy()).cuda()
    W = torch.zeros((gm.N, n * n), dtype=torch.float64, device="cuda")
    E = (0.0, 0.01, 0.03)
    dt = 0.02
    for step in range(2):
        rho, _ = poisson.pair_densities(op, phi_o)
        phi_o, C_o, info_o = sim.step(phi_o, C_o, E, dt, 8)
        info = solver.step(phi, C, W, E, dt, cg_rtol=1e-14, cg_max_it=20000, raise_on_maxit=False)
        torch.cuda.synchronize()
        # the mean fields used by this step: backward error in the oracle's matrices
        Wg = np.empty((om.N, n * n))
        Wg[perm] = W.cpu().numpy()
        assert np.all(sim.ps.residual(Wg, rho) < 1e-12)
        pg = phi.cpu().numpy()
        assert np.linalg.norm(pg - phi_o[perm]) / np.linalg.norm(phi_o) < 1e-10
        cg = C.cpu().numpy()
        assert np.linalg.norm(cg - C_o) / np.linalg.norm(C_o) < 1e-10
        assert abs(info["energy"] - info_o["energy"]) < 1e-10 * abs(info_o["energy"])
        # <sum r_i> at t (scale: the electron count times the box half-width)
        dscale = max(np.max(np.abs(info_o["dipole"])), (na + nb) * 1.0)
        assert np.max(np.abs(np.asarray(info["dipole"]) - info_o["dipole"])) < 1e-10 * dscale
        assert info["krylov_m_used"] == info_o["m_used"]
        assert abs(info["arnoldi_err"] - info_o["arnoldi_err"]) <= 1e-6 * info_o["arnoldi_err"] + 1e-16


def test_singular_density_matrix_is_reported():
    """Two orbitals but only one occupied (a single determinant with C on one
    orbital): gamma is singular and the step returns AFEM_ESINGULAR untouched."""
    import torch
    import paper_2301_02387_gb300 as pkg
    case = (-5.0, 5.0, 2, 2, [((0.0, 0.0, 0.0), 1.0, 1)], 2.0)
    gm = pkg.Mesh(*case)
    X, ml, _ = gm.tables()
    interior = np.arange(gm.N) < gm.n_interior
    phi_h = inputs.lowdin(inputs.molecular_orbitals(X, interior, case[4], 2), ml)
    solver = pkg.MCTDHF(gm, 2, 1, 0, 6)
    phi = torch.from_numpy(phi_h).cuda()
    C = torch.zeros(solver.ci_dim, dtype=torch.complex128, device="cuda")
    C[0] = 1.0
    W = torch.zeros((gm.N, 4), dtype=torch.float64, device="cuda")
    before = phi.clone()
    with pytest.raises(pkg.AfemError) as ei:
        solver.step(phi, C, W, None, 0.02)
    assert ei.value.code == pkg._capi.AFEM_ESINGULAR
    assert torch.equal(phi, before)
