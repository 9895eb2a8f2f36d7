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


# ------------------------------------------------------- Kelly refinement
KELLY_CASE = dict(lo=-8.0, hi=8.0, nc=4, nuclei=[((0.0, 0.0, 0.7), 1.0, 5), ((0.0, 0.0, -0.7), 1.0, 5)])


def test_kelly_face_quadrature_is_exact_for_the_jump():
    """The (p+1)^2-point Gauss rule integrates the squared jump of the normal
    derivative exactly (a polynomial of degree 2p per face direction): the
    indicator of a leaf equals the same sum by a fine midpoint rule."""
    p = 2
    nuc = [(np.array(R), Z, L) for (R, Z, L) in KELLY_CASE["nuclei"]]
    leaves = mesh.balance_leaves({(0, i, j, k) for i in range(4) for j in range(4) for k in range(4)} -
                                 {(0, 1, 1, 1)} | {(1, 2 + a, 2 + b, 2 + c) for a in (0, 1) for b in (0, 1)
                                                    for c in (0, 1)}, 4)
    eta2 = mesh.kelly_indicators(leaves, 4, -8.0, 4.0, p, nuc)
    leaf = (0, 0, 1, 1)   # a coarse leaf beside the refined one (a face with four finer neighbours)
    xi, _ = gll.gll_nodes_weights(p)
    h, c0 = 4.0, np.array([-8.0, -4.0, -4.0])

    def interp_grad(lf, X, d):
        hh = 4.0 / 2 ** lf[0]
        cc = np.array([-8.0 + lf[1] * hh, -8.0 + lf[2] * hh, -8.0 + lf[3] * hh])
        pts = np.array([[cc[0] + hh * xi[a], cc[1] + hh * xi[b], cc[2] + hh * xi[e]]
                        for e in range(p + 1) for b in range(p + 1) for a in range(p + 1)])
        V = -sum(Z / np.linalg.norm(pts - R, axis=1) for (R, Z, _L) in nuc).reshape(p + 1, p + 1, p + 1)
        T = (X - cc) / hh
        M = [gll.lagrange_matrix(xi, T[:, q]) for q in range(3)]
        M[d] = gll.lagrange_deriv_matrix(xi, T[:, d]) / hh
        return np.einsum("cba,ma,mb,mc->m", V, M[0], M[1], M[2])

    tot = 0.0
    n = 80
    g = (np.arange(n) + 0.5) / n
    U, W = np.meshgrid(g, g, indexing="ij")
    for d in range(3):
        for side in (0, 1):
            nb = [leaf[1], leaf[2], leaf[3]]
            nb[d] += 1 if side else -1
            if not 0 <= nb[d] < 4:
                continue
            o = [a for a in range(3) if a != d]
            X = np.zeros((n * n, 3))
            X[:, d] = c0[d] + side * h
            X[:, o[0]] = c0[o[0]] + h * U.ravel()
            X[:, o[1]] = c0[o[1]] + h * W.ravel()
            # the neighbour leaf of each sample point
            J = np.zeros(n * n)
            for m_ in range(n * n):
                pt = X[m_].copy()
                pt[d] += (1e-9 if side else -1e-9)
                nbl = next(lf for lf in leaves
                           if all(-8.0 + lf[q + 1] * 4.0 / 2 ** lf[0] <= pt[q] <= -8.0 + (lf[q + 1] + 1) * 4.0 / 2 ** lf[0]
                                  for q in range(3)))
                J[m_] = interp_grad(leaf, X[m_:m_ + 1], d)[0] - interp_grad(nbl, X[m_:m_ + 1], d)[0]
            tot += np.sum(J * J) * (h / n) ** 2
    assert abs(h / 24.0 * tot - eta2[leaf]) < 2e-3 * eta2[leaf]   # midpoint rule error ~ (1/n)^2


def test_kelly_refinement_properties():
    """No nuclei: nothing refines.  With nuclei: the leaves tile the box, are
    2:1 balanced, reach the level cap exactly at the nuclei, and no leaf below
    the cap keeps an indicator above the threshold; a smaller threshold never
    gives fewer leaves."""
    assert len(mesh.refine_leaves_kelly(3, -6.0, 4.0, 2, [], 0.1, 4)) == 27
    nuc = [(np.array(R), Z, L) for (R, Z, L) in KELLY_CASE["nuclei"]]
    counts = []
    for theta in (1.0, 0.3):
        m = mesh.Mesh(KELLY_CASE["lo"], KELLY_CASE["hi"], KELLY_CASE["nc"], 2, KELLY_CASE["nuclei"], kelly=(theta, 4))
        assert abs(np.sum(m.h ** 3) - 16.0 ** 3) < 1e-9
        lo, hi = m.corner, m.corner + m.h[:, None]
        for a in range(len(m.lev)):
            touch = np.all((lo <= hi[a] + 1e-12) & (hi >= lo[a] - 1e-12), axis=1)
            assert np.all(np.abs(m.lev[touch] - m.lev[a]) <= 1)
        eta2 = mesh.kelly_indicators(set(m.leaf_tuples()), 4, -8.0, 4.0, 2, nuc)
        for lf, e in eta2.items():
            if lf[0] < 4:
                assert e <= theta * theta
            l, i, j, k = lf
            hh = 4.0 / 2 ** l
            cc = np.array([-8.0 + i * hh, -8.0 + j * hh, -8.0 + k * hh])
            if any(np.all((R >= cc) & (R <= cc + hh)) for (R, _Z, _L) in nuc):
                assert l == 4
        counts.append(len(m.lev))
    assert counts[1] >= counts[0]
