"""GPU parity of the two-electron integrals (pq|rs) = sum_f m_f conj(phi_p)
phi_q W^r_s over all support points (Sec. 2, the integrals of Eq. ci_eom with
the mean fields of Eq. mean-field) through afem_two_electron_integrals,
against the oracle's ``MCTDHF.integrals`` on the same orbitals and fields:
the FP64 form within 1e-10, the precision form (the contraction as tcgen05
tensor-core MMAs with TF32 operands split hi/lo and FP64 sums of 32-point
tiles) within 1e-6.  Orbital counts 1..8 cover every accumulator width
(16, 32, 64 columns); the meshes have hanging points, a ragged last tile and
fewer tiles than blocks as well as many more."""
import numpy as np
import pytest

from oracle import fem, mctdhf, mesh as omesh
from paper_2301_02387_gb300 import inputs
from tests._match import assert_close, coord_permutation

pytestmark = pytest.mark.gpu

SMALL = (-8.0, 8.0, 3, 3, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)
Q4 = (-10.0, 10.0, 4, 4, [((0.3, -0.45, 0.7), 1.0, 2), ((-1.1, 0.2, -0.35), 2.0, 2)], 1.5)
LARGER = (-12.0, 12.0, 6, 3, [((0.0, 0.0, 0.0), 8.0, 3), ((1.43, 1.11, 0.0), 1.0, 2),
                              ((-1.43, 1.11, 0.0), 1.0, 2)], 2.0)


def _columns(X, n, seed):
    """Smooth seeded stand-ins for the n^2 real mean-field columns (potential-like
    decay plus a Gaussian bump per column)."""
    rng = np.random.default_rng(seed)
    r = np.sqrt(np.sum(X ** 2, axis=1))
    cols = np.empty((len(X), n * n))
    for c in range(n * n):
        ctr = rng.uniform(-2.0, 2.0, 3)
        amp = rng.uniform(0.2, 1.0)
        cols[:, c] = amp / np.sqrt(1.0 + r ** 2) + rng.uniform(-0.5, 0.5) * np.exp(-0.3 * np.sum((X - ctr) ** 2, axis=1))
    return cols


def _oracle_fields(cols, n):
    """W[r][s] of the oracle from the library's column layout: c < n is |phi_c|^2's
    field; then Re, Im of each pair r < s in row-major order; W_sr = conj(W_rs)."""
    N = cols.shape[0]
    W = np.zeros((n, n, N), dtype=np.complex128)
    for r in range(n):
        W[r, r] = cols[:, r]
    c = n
    for r in range(n):
        for s in range(r + 1, n):
            W[r, s] = cols[:, c] + 1j * cols[:, c + 1]
            W[s, r] = np.conj(W[r, s])
            c += 2
    return W


@pytest.mark.parametrize("case,n", [(SMALL, 1), (SMALL, 2), (SMALL, 3), (Q4, 4), (Q4, 5), (SMALL, 8),
                                    (LARGER, 4), (LARGER, 8)])
def test_integrals_match_oracle(case, n):
    import torch
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    phi_o = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, case[4], n), op.ML)
    cols_o = _columns(om.Xm, n, seed=100 + n)
    sim = mctdhf.MCTDHF(op, n, 1, 0)
    _, eri_o = sim.integrals(phi_o, _oracle_fields(cols_o, n), (0.0, 0.0, 0.0))
    ref = eri_o.reshape(n * n, n * n)
    phi = torch.from_numpy(np.ascontiguousarray(phi_o[perm])).cuda()
    W = torch.from_numpy(np.ascontiguousarray(cols_o[perm])).cuda()
    eri64 = pkg.two_electron_integrals(gm, phi, W, precision=pkg.PREC_FP64)
    torch.cuda.synchronize()
    assert_close(eri64.cpu().numpy(), ref, 1e-10, what="FP64 integrals")
    for _ in range(2):   # two calls in a row reuse the workspace and the tensor memory
        eri32 = pkg.two_electron_integrals(gm, phi, W, precision=pkg.PREC_MIXED)
        torch.cuda.synchronize()
        assert_close(eri32.cpu().numpy(), ref, 1e-6, what="tensor-core integrals")


def test_integrals_argument_checks():
    import torch
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(*SMALL)
    phi = torch.zeros((gm.N, 9), dtype=torch.complex128, device="cuda")
    W = torch.zeros((gm.N, 81), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.AfemError):
        pkg.two_electron_integrals(gm, phi, W)
    phi = torch.zeros((gm.N, 2), dtype=torch.complex128, device="cuda")
    W = torch.zeros((gm.N, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.AfemError):
        pkg.two_electron_integrals(gm, phi, W, precision=7)
