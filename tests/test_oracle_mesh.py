"""Pins for the oracle mesh: refinement rule, 2:1 balance and the hanging-node
("bridged" function) constraints of Sec. 3.1."""
import itertools

import numpy as np
import pytest

from oracle import gll, mesh

H_CASE = dict(lo=-10.0, hi=10.0, nc=4, nuclei=[((0.0, 0.0, 0.0), 1.0, 3)], c=2.0)
OFF_CASE = dict(lo=-8.0, hi=8.0, nc=4, nuclei=[((0.3, -0.45, 0.7), 1.0, 2),
                                             ((-1.1, 0.2, -0.35), 2.0, 3)], c=1.5)


def _mk(case, p):
    return mesh.Mesh(case["lo"], case["hi"], case["nc"], p, case["nuclei"], case["c"])


def test_uniform_mesh_counts():
    m = mesh.Mesh(-1.0, 1.0, 3, 3, [], 2.0)
    assert len(m.lev) == 27
    assert m.nf == (3 * 3 + 1) ** 3
    assert m.n_hanging == 0 and m.N == m.nf
    assert m.boundary.sum() == (3 * 3 + 1) ** 3 - (3 * 3 - 1) ** 3


@pytest.mark.parametrize("case", [H_CASE, OFF_CASE])
def test_leaves_tile_box_and_rule_holds(case):
    m = _mk(case, 1)
    vol = np.sum(m.h ** 3)
    assert abs(vol - (case["hi"] - case["lo"]) ** 3) < 1e-9
    # no leaf remains that the rule would still split
    for q in range(len(m.lev)):
        for (R, _Z, L) in m.nuclei:
            if m.lev[q] < L:
                lo = m.corner[q]
                d = np.maximum(0.0, np.maximum(lo - R, R - (lo + m.h[q])))
                assert np.dot(d, d) > (case["c"] * m.h[q]) ** 2


@pytest.mark.parametrize("case", [H_CASE, OFF_CASE])
def test_two_to_one_balance_brute_force(case):
    m = _mk(case, 1)
    lo, hi = m.corner, m.corner + m.h[:, None]
    n = len(m.lev)
    for a in range(n):
        touch = np.all((lo <= hi[a] + 1e-12) & (hi >= lo[a] - 1e-12), axis=1)
        assert np.all(np.abs(m.lev[touch] - m.lev[a]) <= 1)
    assert m.lev.max() == max(L for (_R, _Z, L) in m.nuclei)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_constraints_reproduce_q_p_polynomials(p):
    m = _mk(OFF_CASE, p)
    assert m.n_hanging > 0
    rng = np.random.default_rng(7)
    coef = rng.standard_normal((p + 1, p + 1, p + 1))
    x, y, z = (m.X[:, a] / 8.0 for a in range(3))

    def g(x, y, z):
        out = np.zeros_like(x)
        for a, b, c in itertools.product(range(p + 1), repeat=3):
            out += coef[a, b, c] * x ** a * y ** b * z ** c
        return out
    gf = g(x, y, z)
    np.testing.assert_allclose(m.C @ gf[m.master_pts], gf, atol=1e-11 * np.abs(gf).max())


@pytest.mark.parametrize("p", [2, 3, 4])
def test_random_fe_function_is_continuous_across_coarse_fine_faces(p):
    """Fine-cell and coarse-cell polynomials of a random FE function agree on
    their shared face or edge (evaluated from float coordinates)."""
    m = _mk(OFF_CASE, p)
    rng = np.random.default_rng(3)
    uf = m.C @ rng.standard_normal(m.N)
    cell_of = {(int(m.lev[q]), *map(int, m.ijk[q])): q for q in range(len(m.lev))}
    hang = np.nonzero(m.hanging)[0]
    checked = 0
    for h in rng.choice(hang, size=min(60, len(hang)), replace=False):
        cells = [cell_of[c] for c in m.containing_cells(h)]
        lmin = min(m.lev[q] for q in cells)
        coarse = [q for q in cells if m.lev[q] == lmin]
        fine = [q for q in cells if m.lev[q] > lmin]
        for qc in coarse:
            for qf in fine:
                lo = np.maximum(m.corner[qc], m.corner[qf])
                hi = np.minimum(m.corner[qc] + m.h[qc], m.corner[qf] + m.h[qf])
                pts = lo + rng.random((5, 3)) * (hi - lo)
                vals = []
                for q in (qc, qf):
                    t = (pts - m.corner[q]) / m.h[q]
                    B = np.einsum("ia,ib,ic->icba",
                                  gll.lagrange_matrix(m.xi, t[:, 0]),
                                  gll.lagrange_matrix(m.xi, t[:, 1]),
                                  gll.lagrange_matrix(m.xi, t[:, 2])).reshape(len(pts), -1)
                    vals.append(B @ uf[m.cell_pts[q]])
                np.testing.assert_allclose(vals[0], vals[1], atol=1e-12)
                checked += 1
    assert checked > 20


def test_boundary_flags():
    m = _mk(H_CASE, 2)
    on = np.any(np.isclose(np.abs(m.Xm), 10.0, atol=1e-12), axis=1)
    assert np.array_equal(on, m.boundary)
