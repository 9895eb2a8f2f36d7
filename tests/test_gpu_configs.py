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
from tests._match import coord_permutation

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
            rel = np.linalg.norm(phi.cpu().numpy() - phi_o[perm]) / np.linalg.norm(phi_o)
            assert rel < 1e-10, (k, rel)
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
