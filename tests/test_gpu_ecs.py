"""GPU parity of exterior complex scaling (afem_mesh_set_ecs; Sec. 4's
absorbing boundary, the reading in ``oracle.fem``) against the oracle's
assembled scaled operators: the one-body operator in FP64 and complex64, the
MCTDHF step (scaled G inside the Arnoldi step, non-Hermitian CI) in both
arithmetic forms, and the argument checks."""
import numpy as np
import pytest

from oracle import fem, mctdhf, mesh as omesh
from paper_2301_02387_gb300 import inputs
from tests._match import assert_close, coord_permutation

pytestmark = pytest.mark.gpu

# (mesh, inner-box half widths): the box faces lie on cell faces
CASES = [
    ((-10.0, 10.0, 10, 3, [((0.0, 0.0, 0.0), 0.0, 0)], 2.0), (6.0, 6.0, 6.0)),            # uniform, Z = 0
    ((-8.0, 8.0, 4, 3, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0), (4.0, 4.0, 4.0)),
    ((-8.0, 8.0, 4, 4, [((0.3, -0.45, 0.7), 1.0, 2), ((-1.1, 0.2, -0.35), 2.0, 2)], 1.5), (4.0, 8.0, 4.0)),
    ((-6.0, 6.0, 3, 2, [((0.0, 0.0, 0.0), 1.0, 1)], 2.0), (2.0, 2.0, 6.0)),
]


def _pair(case, R, theta):
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    op.set_ecs(theta, R)
    pkg.mesh_set_ecs(gm, theta, R)
    X, _, _ = gm.tables()
    return gm, om, op, coord_permutation(X, om.Xm)


@pytest.mark.parametrize("case,R", CASES)
@pytest.mark.parametrize("nvec", [1, 2, 4])
def test_ecs_h1_parity(case, R, nvec):
    """M_L^-1 H1~ with the scaled kinetic term: FP64 within 1e-10, complex64 within 2e-5."""
    import torch
    import paper_2301_02387_gb300 as pkg
    gm, om, op, perm = _pair(case, R, 0.4)
    rng = np.random.default_rng(31)
    xo = rng.standard_normal((om.N, nvec)) + 1j * rng.standard_normal((om.N, nvec))
    E = (0.013, -0.02, 0.031)
    yo = op.h1_apply(xo, E=E)
    x = torch.from_numpy(np.ascontiguousarray(xo[perm])).cuda()
    y = torch.empty_like(x)
    pkg.op_apply(gm, pkg.OP_H1, x, y, E=E)
    torch.cuda.synchronize()
    assert_close(y.cpu().numpy(), yo[perm], 1e-10, what="FP64")
    x32 = x.to(torch.complex64)
    yo32 = op.h1_apply(x32.cpu().numpy().astype(np.complex128)[np.argsort(perm)], E=E)
    y32 = torch.empty_like(x32)
    pkg.op_apply(gm, pkg.OP_H1_C64, x32, y32, E=E)
    torch.cuda.synchronize()
    assert_close(y32.to(torch.complex128).cpu().numpy(), yo32[perm], 2e-5, what="complex64")


def test_ecs_removed_restores_the_operator():
    import torch
    import paper_2301_02387_gb300 as pkg
    case, R = CASES[1]
    gm = pkg.Mesh(*case)
    rng = np.random.default_rng(2)
    x = torch.from_numpy(rng.standard_normal((gm.N, 2)) + 1j * rng.standard_normal((gm.N, 2))).cuda()
    y0, y1, y2 = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    pkg.op_apply(gm, pkg.OP_H1, x, y0)
    pkg.mesh_set_ecs(gm, 0.5, R)
    pkg.op_apply(gm, pkg.OP_H1, x, y1)
    pkg.mesh_set_ecs(gm, 0.0, R)
    pkg.op_apply(gm, pkg.OP_H1, x, y2)
    torch.cuda.synchronize()
    # the scatter adds by atomics, so repeated applies agree to rounding order only
    assert_close(y2.cpu().numpy(), y0.cpu().numpy(), 1e-14, what="unscaled again")
    assert (y1 - y0).abs().max().item() > 1e-3 * y0.abs().max().item()


def test_ecs_argument_checks():
    import torch
    import paper_2301_02387_gb300 as pkg
    case, R = CASES[0]
    gm = pkg.Mesh(*case)
    with pytest.raises(pkg.AfemError):
        pkg.mesh_set_ecs(gm, 0.4, (5.0, 6.0, 6.0))      # x = +-5 cuts cells
    with pytest.raises(pkg.AfemError):
        pkg.mesh_set_ecs(gm, 1.6, R)                    # theta >= pi/2
    with pytest.raises(pkg.AfemError):
        pkg.mesh_set_ecs(gm, 0.4, (6.0, -1.0, 6.0))
    pkg.mesh_set_ecs(gm, 0.4, R)
    x = torch.zeros((gm.N, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(pkg.AfemError):
        pkg.op_apply(gm, pkg.OP_H1_VG, x, torch.empty_like(x), E=(0.0, 0.0, 0.1))


@pytest.mark.parametrize("precision_name", ["fp64", "mixed"])
def test_ecs_mctdhf_step_parity(precision_name):
    """Two steps with the scaled kinetic term (non-Hermitian h_pq and CI
    Hamiltonian) against the oracle: FP64 within 1e-10, the precision form
    within 1e-6."""
    import torch
    import paper_2301_02387_gb300 as pkg
    case, R = CASES[1]
    n, na, nb = 2, 1, 1
    gm, om, op, perm = _pair(case, R, 0.4)
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, case[4], n), op.ML)
    C_o = inputs.initial_ci(n, na, nb, amp=0.1)
    sim = mctdhf.MCTDHF(op, n, na, nb)
    solver = pkg.MCTDHF(gm, n, na, nb, 8)
    prec = pkg.PREC_FP64 if precision_name == "fp64" else pkg.PREC_MIXED
    solver.set_precision(prec)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    C = torch.from_numpy(C_o.copy()).cuda()
    W = torch.zeros((gm.N, n * n), dtype=torch.float64, device="cuda")
    E = (0.0, 0.01, 0.03)
    bar = 1e-10 if precision_name == "fp64" else 1e-6
    for _ in range(2):
        phi_o, C_o, info_o = sim.step(phi_o, C_o, E, 0.02, 8)
        info = solver.step(phi, C, W, E, 0.02, cg_rtol=1e-14, cg_max_it=20000, raise_on_maxit=False)
        torch.cuda.synchronize()
        assert_close(phi.cpu().numpy(), phi_o[perm], bar, what="orbitals")
        assert_close(C.cpu().numpy(), C_o, bar, what="CI vector")
        assert abs(info["energy"] - info_o["energy"]) < bar * abs(info_o["energy"])
    solver.set_imaginary(True)
    with pytest.raises(pkg.AfemError):
        solver.step(phi, C, W, E, 0.02)
    solver.close()
