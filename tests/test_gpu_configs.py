"""GPU parity on the smallest workload as specified end to end: the hydrogen
atom at the origin on [-20,20]^3 (8^3 coarse, Q2, 3 levels; N = 17,213),
one orbital exp(-r^2) with 1e-3 phase noise, 100 field-free steps of
dt = 0.01 by Krylov steps of dimension 8 (Sec. 3.2, the projector with the
frozen orbital of each step), then the Poisson solve of |phi|^2 at rtol 1e-10
(Sec. 3.1, Eq. mean-field).  The oracle runs the same sequence with its
assembled operators; FP64 bar 1e-10 relative, Poisson by backward error."""
import numpy as np
import pytest

from oracle import fem, krylov, mctdhf, mesh as omesh, poisson
from paper_2301_02387_gb300 import inputs
from tests._match import assert_close, coord_permutation, rel_errors

pytestmark = pytest.mark.gpu


def test_hydrogen_q2_propagation_and_poisson():
    import torch
    import paper_2301_02387_gb300 as pkg
    name = "hydrogen_q2"
    w = inputs.WORKLOADS[name]
    gm = pkg.Mesh(*inputs.mesh_args(name))
    om = omesh.Mesh(*inputs.mesh_args(name))
    assert om.N == gm.N == 17213
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    interior = ~om.boundary
    g = inputs.gaussian_orbital(om.Xm, interior)
    phi_o = (g / np.sqrt(np.sum(op.ML * np.abs(g) ** 2)))[:, None]
    sim = mctdhf.MCTDHF.__new__(mctdhf.MCTDHF)
    sim.ops, sim.mesh, sim.n = op, om, 1
    sim.interior = interior.astype(np.float64)
    U0 = np.zeros((1, 1, om.N), dtype=np.complex128)
    E0 = (0.0, 0.0, 0.0)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    assert w["steps"] == 100 and w["m"] == 8 and w["pulse"] is None
    for k in range(w["steps"]):
        cur = phi_o
        phi_o, *_ = krylov.arnoldi_expm(lambda v: sim.G_apply(v, cur, U0, E0), cur, sim.inner, w["m"], w["dt"])
        phi, err, mu, brk = pkg.arnoldi_step(gm, phi, None, w["m"], w["dt"])
        if k in (0, w["steps"] - 1):
            torch.cuda.synchronize()
            assert_close(phi.cpu().numpy(), phi_o[perm], 1e-10, what=f"step {k}")
    pg = np.empty_like(phi_o)
    pg[perm] = phi.cpu().numpy()
    W = torch.zeros((gm.N, 1), dtype=torch.float64, device="cuda")
    it, rel, rc = pkg.poisson_batch(gm, phi, W, rtol=1e-10, max_it=20000)
    assert rc == 0 and rel[0] <= 1e-10
    ps = poisson.PoissonSolver(op)
    rho, _ = poisson.pair_densities(op, pg)
    Wg = np.empty((om.N, 1))
    Wg[perm] = W.cpu().numpy()
    assert ps.residual(Wg, rho)[0] < 2e-10


def test_water_q4_sampled_rows():
    """The water workload's mesh at full size (O + 2 H, [-50,50]^3, 32^3
    coarse, Q4, 6 / 5 levels: 2,560,197 masters) in its launch
    configurations: H1~ on 8 complex orbitals (FP64 and complex64) and the
    stiffness on the 64 columns of its Poisson batch (FP64 and FP32), compared
    on 3,000+ sampled masters (random, every kind of constraint master, and
    those nearest the nuclei) with the oracle's rows formed cell by cell."""
    import torch
    import paper_2301_02387_gb300 as pkg
    from oracle import rows
    name = "water_q4"
    w = inputs.WORKLOADS[name]
    gm = pkg.Mesh(*inputs.mesh_args(name))
    om = omesh.Mesh(*inputs.mesh_args(name))
    assert om.N == gm.N == 2560197
    ro = rows.RowOperators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    rng = np.random.default_rng(51)
    hang = np.nonzero(om.hanging)[0]
    cons = np.unique(om.C.tocsr()[hang].indices)
    near = np.concatenate([np.argsort(np.sum((om.Xm - np.asarray(R)) ** 2, axis=1))[:200]
                           for (R, _Z, _L) in w["nuclei"]])
    R = np.unique(np.concatenate([rng.choice(om.N, 2000, replace=False), rng.choice(cons, 1000, replace=False),
                                  near]))
    lib = torch.from_numpy(inv[R]).cuda()

    def rel(a, b):
        return max(rel_errors(a, b, axis=0))

    n = w["n_orb"]
    phi = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, w["nuclei"], n), ro.ML)
    xo = phi + 0.05 * (rng.standard_normal(phi.shape) + 1j * rng.standard_normal(phi.shape))
    E = (0.03, -0.05, 0.0755)
    yo = ro.h1_rows(R, xo, E=E)
    x = torch.from_numpy(np.ascontiguousarray(xo[perm])).cuda()
    y = torch.empty_like(x)
    pkg.op_apply(gm, pkg.OP_H1, x, y, E=E)
    assert rel(y[lib].cpu().numpy(), yo) < 1e-10
    x32o = xo.astype(np.complex64).astype(np.complex128)
    y32o = ro.h1_rows(R, x32o, E=E)
    x32 = x.to(torch.complex64)
    y32 = torch.empty_like(x32)
    pkg.op_apply(gm, pkg.OP_H1_C64, x32, y32, E=E)
    assert rel(y32[lib].to(torch.complex128).cpu().numpy(), y32o) < 2e-5
    del x, y, x32, y32
    so = rng.standard_normal((om.N, n * n)).astype(np.float32).astype(np.float64)
    yso = ro.stiffness_rows(R, so)
    s = torch.from_numpy(np.ascontiguousarray(so[perm])).cuda()
    ys = torch.empty_like(s)
    pkg.op_apply(gm, pkg.OP_STIFF, s, ys)
    assert rel(ys[lib].cpu().numpy(), yso) < 1e-10
    s32 = s.float()
    ys32 = torch.empty_like(s32)
    pkg.op_apply(gm, pkg.OP_STIFF_F32, s32, ys32)
    assert rel(ys32[lib].double().cpu().numpy(), yso) < 2e-5
