"""Batching form: the FP32 cell passes of several meshes (uneven sizes,
degrees 1..4) in one persistent launch must give each instance what the
single-instance afem_op_apply gives it (up to the order of the float atomic
sums), also when replayed from the captured graph and after the fields or
buffers change; and every instance is compared with the oracle's assembled
operators (Sec. 3.1) directly, odd orbital counts included."""
import numpy as np
import pytest

from oracle import fem, mesh as omesh
from tests._match import assert_close, coord_permutation

pytestmark = pytest.mark.gpu

CASES = [
    (-6.0, 6.0, 2, 2, [((0.0, 0.0, 0.0), 1.0, 2)], 2.0),
    (-8.0, 8.0, 3, 4, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0),
    (-5.0, 5.0, 2, 3, [((0.3, -0.2, 0.1), 3.0, 2)], 1.5),
    (-4.0, 4.0, 2, 1, [((0.5, 0.5, 0.5), 1.0, 1)], 2.0),
]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _meshes():
    from paper_2301_02387_gb300 import Mesh
    return [Mesh(*c) for c in CASES]


def test_batched_orbital_operator_matches_single_instance():
    import torch
    import paper_2301_02387_gb300 as pkg
    meshes = _meshes()
    batch = pkg.Batch(meshes)
    rng = np.random.default_rng(3)
    nvec = [2, 4, 2, 2]
    xs = [torch.from_numpy((rng.standard_normal((m.N, k)) + 1j * rng.standard_normal((m.N, k)))
                           .astype(np.complex64)).cuda() for m, k in zip(meshes, nvec)]
    E = [(0.01, -0.02, 0.03), (0.0, 0.0, 0.05), (0.02, 0.0, 0.0), (0.0, 0.01, 0.0)]
    ref = []
    for m, x, e in zip(meshes, xs, E):
        y = torch.empty_like(x)
        pkg.op_apply(m, pkg.OP_H1_C64, x, y, E=e)
        ref.append(y)
    for graph in (False, True, True):
        ys = [torch.full_like(x, float("nan")) for x in xs]
        batch.apply(pkg.OP_H1_C64, xs, ys, E=E, graph=graph)
        torch.cuda.synchronize()
        for y, r in zip(ys, ref):
            assert _rel(y.cpu().numpy(), r.cpu().numpy()) < 1e-6
    t = batch.tuning()
    assert t["tuned"] and t["count"] == len(meshes)
    assert (t["block"], t["grid"]) in [(b, g) for b, g, _ in t["candidates"]]
    # new fields and new output buffers, same graph: the device table is re-uploaded
    E2 = [(0.0, 0.0, -0.04)] * len(meshes)
    ys = [torch.zeros_like(x) for x in xs]
    batch.apply(pkg.OP_H1_C64, xs, ys, E=E2, graph=True)
    torch.cuda.synchronize()
    for m, x, y in zip(meshes, xs, ys):
        r = torch.empty_like(x)
        pkg.op_apply(m, pkg.OP_H1_C64, x, r, E=E2[0])
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), r.cpu().numpy()) < 1e-6
    batch.close()


def test_batched_stiffness_matches_single_instance():
    import torch
    import paper_2301_02387_gb300 as pkg
    meshes = _meshes()
    batch = pkg.Batch(meshes)
    rng = np.random.default_rng(4)
    ks = [4, 16, 8, 4]
    xs = [torch.from_numpy(rng.standard_normal((m.N, k)).astype(np.float32)).cuda() for m, k in zip(meshes, ks)]
    ys = [torch.empty_like(x) for x in xs]
    for graph in (True, True):
        batch.apply(pkg.OP_STIFF_F32, xs, ys, graph=graph)
        torch.cuda.synchronize()
        for m, x, y in zip(meshes, xs, ys):
            r = torch.empty_like(x)
            pkg.op_apply(m, pkg.OP_STIFF_F32, x, r)
            torch.cuda.synchronize()
            assert _rel(y.cpu().numpy(), r.cpu().numpy()) < 1e-6
    batch.close()


def test_batch_rejects_bad_arguments():
    import torch
    import paper_2301_02387_gb300 as pkg
    meshes = _meshes()[:2]
    batch = pkg.Batch(meshes)
    xs = [torch.zeros((m.N, 4), dtype=torch.complex64, device="cuda") for m in meshes]
    with pytest.raises(pkg.AfemError):
        batch.apply(pkg.OP_H1_C64, xs, xs)   # aliased in/out
    xr = [torch.zeros((m.N, 4), dtype=torch.float32, device="cuda") for m in meshes]
    with pytest.raises(pkg.AfemError):
        batch.apply(pkg.OP_STIFF, xr, [torch.empty_like(x) for x in xr])   # not a batched kind
    batch.close()


@pytest.mark.parametrize("nvec", [[1, 3, 2, 5], [2, 4, 6, 8], [7, 1, 1, 3]])
def test_batched_instances_match_oracle(nvec):
    """Each instance of the batch against the oracle's assembled operators:
    y_i = M_L^-1 H1~(E_i) x_i (complex64; odd orbital counts run the
    per-instance schedule, even ones may run the persistent launch) and the
    stiffness on 3, 4, 5 or 12 real columns; inputs rounded to float32 on both
    sides; 2e-5 relative per vector and per entry (float32 rounding times the
    operator norm, the bar of the single-instance tests)."""
    import torch
    import paper_2301_02387_gb300 as pkg
    meshes = _meshes()
    rng = np.random.default_rng(sum(nvec))
    E = [(0.01, -0.02, 0.03), (0.0, 0.0, 0.05), (0.02, 0.0, 0.0), (0.0, 0.01, 0.0)]
    orc, perms = [], []
    for m, c in zip(meshes, CASES):
        om = omesh.Mesh(*c)
        X, _, _ = m.tables()
        perms.append(coord_permutation(X, om.Xm))
        orc.append((om, fem.Operators(om)))
    batch = pkg.Batch(meshes)
    xo = []
    for (om, op), k in zip(orc, nvec):
        x = (rng.standard_normal((om.N, k)) + 1j * rng.standard_normal((om.N, k))).astype(np.complex64)
        xo.append(x.astype(np.complex128))
    xs = [torch.from_numpy(np.ascontiguousarray(x[pm]).astype(np.complex64)).cuda() for x, pm in zip(xo, perms)]
    for graph in (False, True):
        ys = [torch.full_like(x, float("nan")) for x in xs]
        batch.apply(pkg.OP_H1_C64, xs, ys, E=E, graph=graph)
        torch.cuda.synchronize()
        for (om, op), x, y, pm, e in zip(orc, xo, ys, perms, E):
            x = x.copy()
            x[om.boundary] = 0.0
            assert_close(y.to(torch.complex128).cpu().numpy(), op.h1_apply(x, E=e)[pm], 2e-5, axis=0,
                         what=f"H1 instance N={om.N}")
    ks = [3 + (k % 2), 4, 5, 12]
    so = [rng.standard_normal((om.N, k)).astype(np.float32).astype(np.float64) for (om, _), k in zip(orc, ks)]
    ss = [torch.from_numpy(np.ascontiguousarray(x[pm])).float().cuda() for x, pm in zip(so, perms)]
    ys = [torch.empty_like(x) for x in ss]
    batch.apply(pkg.OP_STIFF_F32, ss, ys, graph=True)
    torch.cuda.synchronize()
    for (om, op), x, y, pm in zip(orc, so, ys, perms):
        assert_close(y.double().cpu().numpy(), op.stiffness_apply(x)[pm], 2e-5, axis=0,
                     what=f"stiffness instance N={om.N}")
    t = batch.tuning()
    assert t["tuned"]
    if any(2 * k % 4 for k in nvec):
        assert t["block"] == 0   # odd orbital counts: the per-instance schedule
    batch.close()
