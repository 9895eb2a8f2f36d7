"""Kernel-class event timing of the library (afem_profile_*): the Arnoldi
Gram-Schmidt class records one call per pass with the stated FP64 work."""
import numpy as np
import pytest

from oracle import mesh as omesh
from paper_2301_02387_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_gram_schmidt_class_counts_calls_and_work():
    import torch
    import paper_2301_02387_gb300 as pkg
    case = (-6.0, 6.0, 2, 2, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)
    gm = pkg.Mesh(*case)
    X, ml, _ = gm.tables()
    n, m = 2, 5
    interior = np.arange(gm.N) < gm.n_interior
    phi = inputs.lowdin(inputs.molecular_orbitals(X, interior, case[4], n), ml)
    phi_t = torch.from_numpy(phi).cuda()
    U = torch.zeros((gm.N, n, n), dtype=torch.complex128, device="cuda")
    for c in range(pkg.PROF_COUNT):
        pkg.profile_read(c, reset=True)
    pkg.profile_enable(True)
    try:
        for prec in (pkg.PREC_FP64, pkg.PREC_MIXED):
            pkg.arnoldi_step(gm, phi_t, U, m, 0.01, E=(0.0, 0.0, 0.01), precision=prec)
        torch.cuda.synchronize()
    finally:
        pkg.profile_enable(False)
    ms, calls, work = pkg.profile_read(pkg.PROF_GS, reset=True)
    # two forms x m vectors x (projector/inner-product pass + update pass)
    assert calls == 2 * m * 2
    E = gm.n_interior * n
    # inner-product pass 8 (j+1) flops per element, update 8 (j+1) + 4 (the new norm)
    expect = 2 * sum(E * (16.0 * (j + 1) + 4.0) for j in range(m))
    assert work == pytest.approx(expect, rel=1e-12)
    assert ms > 0.0
    ms_c, calls_c, work_c = pkg.profile_read(pkg.PROF_GCELL32, reset=True)
    assert calls_c == m and ms_c > 0.0 and work_c == pytest.approx(m * gm.N * 8.0 * n * (2 + n))
    ms_f, calls_f, _ = pkg.profile_read(pkg.PROF_CELL64, reset=True)
    assert calls_f == m and ms_f > 0.0
