"""Pins of the row-wise oracle (`oracle/rows.py`): the rows it forms cell by
cell equal those of the globally assembled operators (a different route: one
sparse assembly of C^T A_f C), and on their own they satisfy the identities of
Sec. 3.1's discretisation: A 1 = 0, A x_k = 0 at interior masters, and
A x^2 = -2 M_L at masters whose support stays off the box surface (GLL
quadrature integrates these exactly), with M_L summing to the box volume."""
import numpy as np
import pytest

from oracle import fem, mesh as omesh, rows

CASES = [
    (-8.0, 8.0, 3, 2, [((0.3, -0.45, 0.7), 1.0, 2), ((-1.1, 0.2, -0.35), 2.0, 2)], 1.5),
    (-6.0, 6.0, 2, 3, [((0.0, 0.0, 0.0), 8.0, 1), ((1.4311, 1.1081, 0.0), 1.0, 1)], 2.0),
    (-8.0, 8.0, 3, 4, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0),
    (-6.0, 6.0, 2, 1, [((0.5, 0.5, 0.5), 8.0, 3)], 1.0),
]


def _sample(om, rng, k=300):
    """Random masters plus every master that constrains a hanging point."""
    C = om.C.tocsr()
    hang = np.nonzero(om.hanging)[0]
    cons = np.unique(C[hang].indices) if len(hang) else np.zeros(0, dtype=np.int64)
    pick = rng.choice(om.N, size=min(k, om.N), replace=False)
    return np.unique(np.concatenate([pick, cons[:k]]))


@pytest.mark.parametrize("case", CASES)
def test_rows_equal_assembled_operators(case):
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    ro = rows.RowOperators(om)
    rng = np.random.default_rng(3)
    R = _sample(om, rng)
    np.testing.assert_allclose(ro.ML, op.ML, rtol=1e-14, atol=0)
    x = rng.standard_normal((om.N, 3))
    yA = op.stiffness_apply(x)[R]
    np.testing.assert_allclose(ro.stiffness_rows(R, x), yA, rtol=0, atol=1e-13 * np.abs(yA).max())
    z = rng.standard_normal((om.N, 2)) + 1j * rng.standard_normal((om.N, 2))
    E = (0.013, -0.02, 0.031)
    yH = op.h1_apply(z, E=E)[R]
    np.testing.assert_allclose(ro.h1_rows(R, z, E=E), yH, rtol=0, atol=1e-13 * np.abs(yH).max())


@pytest.mark.parametrize("case", CASES[:3])
def test_rows_reproduce_polynomial_identities(case):
    om = omesh.Mesh(*case)
    ro = rows.RowOperators(om)
    X = om.Xm
    assert abs(ro.ML.sum() - (om.hi - om.lo) ** 3) < 1e-10 * (om.hi - om.lo) ** 3
    rng = np.random.default_rng(4)
    R = _sample(om, rng)
    one = np.ones(om.N)
    assert np.abs(ro.stiffness_rows(R, one)).max() < 1e-12
    inner = R[ro.interior[R]]
    lin = ro.stiffness_rows(inner, X)
    assert np.abs(lin).max() < 1e-11 * np.abs(X).max()
    if om.p >= 2:
        # masters none of whose support cells (those carrying i or a hanging point
        # that i constrains) touches the box surface
        touch = np.any((np.abs(om.corner - om.lo) < 1e-12) | (np.abs(om.corner + om.h[:, None] - om.hi) < 1e-12),
                       axis=1)
        CT = ro.CT
        away = []
        for i in inner:
            pts = CT.indices[CT.indptr[i]:CT.indptr[i + 1]]
            cells = np.concatenate([ro.inc_cell[ro.inc_ptr[p]:ro.inc_ptr[p + 1]] for p in pts])
            if not touch[cells].any():
                away.append(i)
        away = np.array(away)
        assert len(away) > 10
        for k in range(3):
            q = ro.stiffness_rows(away, X[:, k] ** 2)
            np.testing.assert_allclose(q, -2.0 * ro.ML[away], rtol=1e-10, atol=0)
