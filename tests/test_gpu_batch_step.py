"""GPU parity of the batching form at the level of the time step
(afem_batch_stepper_*): uneven instances -- different meshes, degrees 2..4,
orbital counts (odd and even), electron counts, fields and arithmetic forms,
two of them sharing one mesh -- stepped together, each compared after every
batched step with the oracle's MCTDHF step of that instance (Sec. 2,
Sec. 3.2): FP64 instances within 1e-10, precision-form instances within 1e-6,
over enough calls to pass through the stream-count tuning and run on its
choice.  Also the argument checks."""
import numpy as np
import pytest

from oracle import fem, mctdhf, mesh as omesh
from paper_2301_02387_gb300 import inputs
from tests._match import assert_close, coord_permutation

pytestmark = pytest.mark.gpu

H2 = (-6.0, 6.0, 3, 2, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)
INSTANCES = [
    # (mesh, n_orb, n_alpha, n_beta, field, mixed form)
    (H2, 2, 1, 1, (0.0, 0.01, 0.03), False),
    ((-6.0, 6.0, 2, 3, [((0.0, 0.0, 0.0), 3.0, 2), ((1.2, 0.9, 0.0), 1.0, 1)], 2.0), 3, 2, 1,
     (0.02, 0.0, -0.01), False),
    ((-8.0, 8.0, 2, 4, [((0.3, -0.45, 0.7), 1.0, 1), ((-1.1, 0.2, -0.35), 2.0, 1)], 1.5), 4, 2, 1,
     (0.0, 0.0, 0.05), True),
    (H2, 1, 1, 0, (0.03, 0.0, 0.0), True),   # shares the first instance's mesh
]


def test_batched_steps_match_oracle_per_instance():
    import torch
    import paper_2301_02387_gb300 as pkg
    meshes, pairs, sims, solvers, states, orc = {}, [], [], [], [], []
    for k, (case, n, na, nb, E, mixed) in enumerate(INSTANCES):
        key = repr(case)
        if key not in meshes:
            gm = pkg.Mesh(*case)
            om = omesh.Mesh(*case)
            op = fem.Operators(om)
            X, _, _ = gm.tables()
            meshes[key] = (gm, om, op, coord_permutation(X, om.Xm))
        gm, om, op, perm = meshes[key]
        phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, case[4], n), op.ML)
        C_o = inputs.initial_ci(n, na, nb, amp=0.1)
        sims.append(mctdhf.MCTDHF(op, n, na, nb))
        orc.append([phi_o, C_o])
        solver = pkg.MCTDHF(gm, n, na, nb, 8)
        solver.set_precision(pkg.PREC_MIXED if mixed else pkg.PREC_FP64)
        solvers.append(solver)
        states.append((torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda(),
                       torch.from_numpy(C_o.copy()).cuda(),
                       torch.zeros((gm.N, n * n), dtype=torch.float64, device="cuda")))
        pairs.append(perm)
    batch = pkg.BatchStepper(solvers)
    dt = 0.02
    Es = [inst[4] for inst in INSTANCES]
    ncand = None
    for step in range(6):   # cold call, one call per candidate (1, 2, 4 streams), then the choice
        infos = batch.step([s[0] for s in states], [s[1] for s in states], [s[2] for s in states], Es, dt,
                           cg_rtol=1e-14, cg_max_it=20000, raise_on_maxit=False)
        torch.cuda.synchronize()
        for k, (case, n, na, nb, E, mixed) in enumerate(INSTANCES):
            phi_o, C_o, info_o = sims[k].step(orc[k][0], orc[k][1], E, dt, 8)
            orc[k] = [phi_o, C_o]
            bar = 1e-6 if mixed else 1e-10
            phi, C, _ = states[k]
            assert_close(phi.cpu().numpy(), phi_o[pairs[k]], bar, what=f"instance {k} orbitals, step {step}")
            assert_close(C.cpu().numpy(), C_o, bar, what=f"instance {k} CI vector, step {step}")
            assert abs(infos[k]["energy"] - info_o["energy"]) < bar * abs(info_o["energy"])
        tun = batch.tuning()
        ncand = len(tun["candidates"])
    assert ncand == 3 and tun["streams"] in (1, 2, 4)
    assert all(ms > 0.0 for _, ms in tun["candidates"])
    batch.close()


def test_batch_stepper_argument_checks():
    import torch
    import paper_2301_02387_gb300 as pkg
    lib = pkg.load_library()
    import ctypes
    h = ctypes.c_void_p()
    assert lib.afem_batch_stepper_create(None, 0, ctypes.byref(h)) == pkg._capi.AFEM_EINVAL
    gm = pkg.Mesh(*H2)
    solver = pkg.MCTDHF(gm, 2, 1, 1, 8)
    batch = pkg.BatchStepper([solver])
    phi = torch.zeros((gm.N, 2), dtype=torch.complex128, device="cuda")
    C = torch.zeros(solver.ci_dim, dtype=torch.complex128, device="cuda")
    W = torch.zeros((gm.N, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.AfemError):
        batch.step([phi], [C], [W], None, -1.0)
    pkg.profile_enable(True)
    try:
        with pytest.raises(pkg.AfemError):
            batch.step([phi], [C], [W], None, 0.01)
    finally:
        pkg.profile_enable(False)
    batch.close()
