"""GPU parity of afem_op_apply against the oracle's assembled operators
(Sec. 3.1; Eq. discretized_eom for H1~).  FP64 bar: 1e-10 relative per vector."""
import numpy as np
import pytest

from oracle import fem, mesh as omesh
from tests._match import coord_permutation, rel_errors

pytestmark = pytest.mark.gpu

CASES = [
    # (lo, hi, nc, p, nuclei, c): several tiles, hanging faces/edges, ragged counts
    (-10.0, 10.0, 4, 2, [((0.0, 0.0, 0.0), 1.0, 3)], 2.0),
    (-8.0, 8.0, 4, 3, [((0.3, -0.45, 0.7), 1.0, 2), ((-1.1, 0.2, -0.35), 2.0, 3)], 1.5),
    (-8.0, 8.0, 3, 4, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0),
    (-6.0, 6.0, 2, 1, [((0.5, 0.5, 0.5), 8.0, 3)], 1.0),
    (-3.0, 3.0, 1, 2, [], 2.0),   # a single cell: no hanging nodes, all but one node on the surface
]


def _pair(case):
    from paper_2301_02387_gb300 import Mesh
    lo, hi, nc, p, nuclei, c = case
    gm = Mesh(lo, hi, nc, p, nuclei, c)
    om = omesh.Mesh(lo, hi, nc, p, nuclei, c)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    return gm, om, fem.Operators(om), perm


def _relerr(a, b):
    """Worst column of: the L2 relative error and the largest entry error over
    the column's largest reference entry (the per-entry check)."""
    return max(rel_errors(a, b, axis=0))


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nvec", [1, 3])
def test_h1_apply_parity(case, nvec):
    import torch
    from paper_2301_02387_gb300 import op_apply, OP_H1
    gm, om, op, perm = _pair(case)
    rng = np.random.default_rng(11)
    xo = rng.standard_normal((om.N, nvec)) + 1j * rng.standard_normal((om.N, nvec))
    E = (0.013, -0.02, 0.031)
    yo = op.h1_apply(xo, E=E)
    x = torch.from_numpy(np.ascontiguousarray(xo[perm])).cuda()
    y = torch.empty_like(x)
    op_apply(gm, OP_H1, x, y, E=E)
    torch.cuda.synchronize()
    yg = y.cpu().numpy()
    assert _relerr(yg, yo[perm]) < 1e-10


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nvec", [1, 5, 16])
def test_stiffness_apply_parity(case, nvec):
    import torch
    from paper_2301_02387_gb300 import op_apply, OP_STIFF
    gm, om, op, perm = _pair(case)
    rng = np.random.default_rng(5)
    xo = rng.standard_normal((om.N, nvec))
    yo = op.stiffness_apply(xo)
    x = torch.from_numpy(np.ascontiguousarray(xo[perm])).cuda()
    y = torch.empty_like(x)
    op_apply(gm, OP_STIFF, x, y)
    torch.cuda.synchronize()
    assert _relerr(y.cpu().numpy(), yo[perm]) < 1e-10


def test_op_apply_rejects_bad_arguments():
    import torch
    from paper_2301_02387_gb300 import Mesh, op_apply, OP_H1, AfemError
    gm = Mesh(-3.0, 3.0, 2, 2, [], 2.0)
    x = torch.zeros((gm.N, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(AfemError):
        op_apply(gm, 99, x, torch.empty_like(x))   # not an operator kind
    with pytest.raises(AfemError):
        op_apply(gm, OP_H1, x, x)


# 3: scalar-lane kernel; 4, 8, 12, 16: four-lane kernels with 1..4 quads per node,
# whose work items group up to floor(256 / ((p+1)^3 quads)) cells (ragged last
# group on these meshes)
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nvec", [3, 4, 8, 12, 16])
# four-lane: node-per-thread / line-ordered / column-pair lines (1, 2, 4 quads)
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_stiffness_f32_within_fp32_tolerance(case, nvec, variant):
    """Precision form of the stiffness: relative error a few float32 ulps x operator norm."""
    import torch
    from paper_2301_02387_gb300 import op_apply, OP_STIFF_F32, mesh_set_option, OPT_CELL32_VARIANT
    gm, om, op, perm = _pair(case)
    mesh_set_option(gm, OPT_CELL32_VARIANT, variant)
    rng = np.random.default_rng(9)
    xo = rng.standard_normal((om.N, nvec)).astype(np.float32).astype(np.float64)
    yo = op.stiffness_apply(xo)
    x = torch.from_numpy(np.ascontiguousarray(xo[perm])).float().cuda()
    y = torch.empty_like(x)
    op_apply(gm, OP_STIFF_F32, x, y)
    torch.cuda.synchronize()
    assert _relerr(y.double().cpu().numpy(), yo[perm]) < 2e-5


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nvec", [1, 2, 4, 6, 8])   # 1: scalar-lane kernel; 2..8: 1..4 quads per node
@pytest.mark.parametrize("variant", [0, 1])
def test_h1_c64_within_fp32_tolerance(case, nvec, variant):
    import torch
    from paper_2301_02387_gb300 import op_apply, OP_H1_C64, mesh_set_option, OPT_CELL32_VARIANT
    gm, om, op, perm = _pair(case)
    mesh_set_option(gm, OPT_CELL32_VARIANT, variant)
    rng = np.random.default_rng(12)
    xo = (rng.standard_normal((om.N, nvec)) + 1j * rng.standard_normal((om.N, nvec))).astype(np.complex64)
    xo = xo.astype(np.complex128)
    E = (0.013, -0.02, 0.031)
    yo = op.h1_apply(xo, E=E)
    x = torch.from_numpy(np.ascontiguousarray(xo[perm])).to(torch.complex64).cuda()
    y = torch.empty_like(x)
    op_apply(gm, OP_H1_C64, x, y, E=E)
    torch.cuda.synchronize()
    assert _relerr(y.to(torch.complex128).cpu().numpy(), yo[perm]) < 2e-5


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nvec", [1, 4])
def test_h1_velocity_gauge_parity(case, nvec):
    """AFEM_OP_H1_VG (Sec. 2: -i A . grad, skew-symmetric form) against the
    oracle's H1~(A): FP64 within 1e-10 per vector and per entry, complex64
    within 2e-5 (on inputs rounded to complex64)."""
    import torch
    from paper_2301_02387_gb300 import op_apply, OP_H1_VG, OP_H1_VG_C64
    gm, om, op, perm = _pair(case)
    rng = np.random.default_rng(13)
    xo = rng.standard_normal((om.N, nvec)) + 1j * rng.standard_normal((om.N, nvec))
    A = (0.4, -0.25, 0.6)
    yo = op.h1_apply(xo, A=A)
    x = torch.from_numpy(np.ascontiguousarray(xo[perm])).cuda()
    y = torch.empty_like(x)
    op_apply(gm, OP_H1_VG, x, y, E=A)
    torch.cuda.synchronize()
    assert _relerr(y.cpu().numpy(), yo[perm]) < 1e-10
    x32o = xo.astype(np.complex64).astype(np.complex128)
    y32o = op.h1_apply(x32o, A=A)
    x32 = torch.from_numpy(np.ascontiguousarray(x32o[perm])).to(torch.complex64).cuda()
    y32 = torch.empty_like(x32)
    op_apply(gm, OP_H1_VG_C64, x32, y32, E=A)
    torch.cuda.synchronize()
    assert _relerr(y32.to(torch.complex128).cpu().numpy(), y32o[perm]) < 2e-5


def test_h1_and_stiffness_on_a_kelly_mesh():
    """The operators on a mesh refined by Kelly's indicator (Sec. 3.1) against
    the oracle's assembled ones on its own Kelly mesh (the same leaves)."""
    import torch
    from paper_2301_02387_gb300 import Mesh, op_apply, OP_H1, OP_STIFF
    case = (-8.0, 8.0, 4, 3, [((0.0, 0.0, 0.7), 1.0, 5), ((0.0, 0.0, -0.7), 1.0, 5)], 2.0)
    gm = Mesh(*case, kelly=(0.3, 4))
    om = omesh.Mesh(*case, kelly=(0.3, 4))
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    rng = np.random.default_rng(17)
    xo = rng.standard_normal((om.N, 2)) + 1j * rng.standard_normal((om.N, 2))
    E = (0.01, 0.02, -0.03)
    x = torch.from_numpy(np.ascontiguousarray(xo[perm])).cuda()
    y = torch.empty_like(x)
    op_apply(gm, OP_H1, x, y, E=E)
    torch.cuda.synchronize()
    assert _relerr(y.cpu().numpy(), op.h1_apply(xo, E=E)[perm]) < 1e-10
    so = rng.standard_normal((om.N, 4))
    s = torch.from_numpy(np.ascontiguousarray(so[perm])).cuda()
    ys = torch.empty_like(s)
    op_apply(gm, OP_STIFF, s, ys)
    torch.cuda.synchronize()
    assert _relerr(ys.cpu().numpy(), op.stiffness_apply(so)[perm]) < 1e-10
