"""Adaptive octree mesh, global support points and hanging-node constraints.

Sec. 3.1: the box is first covered by coarse uniform cubes; cells near the
nuclei are repeatedly halved.  The paper drives the refinement by Kelly's
indicator on the nuclear Coulomb potential (`refine_leaves_kelly`, with a
threshold and a smallest cell size); the workloads use a geometric rule:
a leaf of level l is split while some nucleus a with l < L_a lies within
distance c * h_l of the closed cell.  Either way the leaves are 2:1 balanced
across faces, edges and vertices.

The finite-element space is the conforming Q_p space on the leaves: the cell
basis functions are tensor products of 1D Lagrange polynomials through the
GLL points (Sec. 3.1), and continuity across a coarse/fine interface is
enforced by the paper's "bridged" functions.  Concretely, a support point
that is not a node of the coarsest leaves whose closures contain it is a
*hanging* point: its value is that coarse leaf's polynomial evaluated there.
All other support points are *masters* (the global unknowns).  The constraint
matrix C (full points x masters) has identity rows for masters and
interpolation rows for hanging points.

Test infrastructure only (see the package docstring).
"""
import itertools

import numpy as np
import scipy.sparse as sp

from . import gll

KEY_BITS = 40                # fractional bits of the integer point keys (keys stay below 2^62)
_DIRS26 = [d for d in itertools.product((-1, 0, 1), repeat=3) if d != (0, 0, 0)]


def _box_dist2(lo_corner, h, R):
    """Squared distance from point R to the closed box [lo_corner, lo_corner + h]^3."""
    d2 = 0.0
    for ax in range(3):
        a = lo_corner[ax]
        b = a + h
        if R[ax] < a:
            d2 += (a - R[ax]) ** 2
        elif R[ax] > b:
            d2 += (R[ax] - b) ** 2
    return d2


def refine_leaves(nc, lo, h0, nuclei, c):
    """Leaves (level, i, j, k) after the geometric refinement rule.

    nuclei: list of (R (3,), Z, L) with L the number of refinement levels.
    A leaf of level l is split if, for some nucleus with l < L,
    dist(R, closed cell)^2 <= (c h_l)^2.  Repeats until nothing splits.
    """
    leaves = set(itertools.product([0], range(nc), range(nc), range(nc)))
    while True:
        new = set()
        split_any = False
        for (l, i, j, k) in leaves:
            h = h0 / 2 ** l
            corner = (lo + i * h, lo + j * h, lo + k * h)
            split = False
            for (R, _Z, L) in nuclei:
                if l < L and _box_dist2(corner, h, R) <= (c * h) ** 2:
                    split = True
                    break
            if split:
                split_any = True
                for a, b, d in itertools.product((0, 1), repeat=3):
                    new.add((l + 1, 2 * i + a, 2 * j + b, 2 * k + d))
            else:
                new.add((l, i, j, k))
        leaves = new
        if not split_any:
            return leaves


def _find_leaf(leafset, l, i, j, k):
    """The leaf that contains the level-l cell (i, j, k), if it is that cell or an ancestor."""
    for l2 in range(l, -1, -1):
        s = l - l2
        key = (l2, i >> s, j >> s, k >> s)
        if key in leafset:
            return key
    return None


def balance_leaves(leaves, nc):
    """2:1 balance over faces, edges and vertices: touching leaves differ by <= 1 level.

    A leaf of level l is touched by a coarser leaf only if that coarser leaf
    contains one of the 26 same-level neighbour cells of l; if its level is
    below l - 1 it is split.  Repeats until stable.
    """
    leafset = set(leaves)
    while True:
        to_split = set()
        for (l, i, j, k) in leafset:
            if l < 2:
                continue
            n = nc << l
            for dx, dy, dz in _DIRS26:
                a, b, d = i + dx, j + dy, k + dz
                if not (0 <= a < n and 0 <= b < n and 0 <= d < n):
                    continue
                f = _find_leaf(leafset, l, a, b, d)
                if f is not None and f[0] < l - 1:
                    to_split.add(f)
        if not to_split:
            return leafset
        for (l, i, j, k) in to_split:
            leafset.remove((l, i, j, k))
            for a, b, d in itertools.product((0, 1), repeat=3):
                leafset.add((l + 1, 2 * i + a, 2 * j + b, 2 * k + d))


# ------------------------------------------------------- Kelly refinement
# mean of 1/|r| over the unit cube centred at the origin: 3 ln(2 + sqrt 3) - pi/2
_CUBE_MEAN_INV_R = 3.0 * np.log(2.0 + np.sqrt(3.0)) - np.pi / 2.0


def _coulomb(X, nuclei, s):
    """V = -sum Z / |x - R| at the points X; at a point on a nucleus the mean of
    1/|r| over a cube of side s (the point's GLL volume) replaces 1/|r|."""
    V = np.zeros(len(X))
    for (R, Z, _L) in nuclei:
        d = np.linalg.norm(X - R[None, :], axis=1)
        on = d <= 1e-10
        V[~on] -= Z / d[~on]
        V[on] -= Z * _CUBE_MEAN_INV_R / s[on]
    return V


def _contains_nucleus(corner, h, nuclei):
    return any(_box_dist2(corner, h, R) == 0.0 for (R, _Z, _L) in nuclei)


def kelly_indicators(leafset, nc, lo, h0, p, nuclei):
    """eta_K^2 of every leaf: (h_K / 24) sum over its faces F of int_F [d_n V_h]^2.

    Sec. 3.1: Kelly's indicator on the Coulomb potential of the nuclei.  V_h is
    the cellwise interpolant of V = -sum Z_a / |r - R_a| at the cell's GLL
    nodes; [d_n V_h] the jump of its normal derivative between the cell and
    the leaf across each (sub)face (a coarser leaf covers the whole face, four
    finer leaves a quarter each; at a node on a nucleus 1/|r| is replaced by
    its mean over a cube of the node's GLL volume, as for the potential), integrated by the (p+1) x (p+1)
    Gauss-Legendre rule of the (sub)face; faces on the box surface carry no
    jump.  A leaf whose closed box contains a nucleus gets +inf (V is
    unbounded there).  Returns {leaf: eta^2}.
    """
    xi, w = gll.gll_nodes_weights(p)
    wcube = np.array([np.cbrt(w[a] * w[b] * w[cc])
                      for cc in range(p + 1) for b in range(p + 1) for a in range(p + 1)])
    gx, gw = np.polynomial.legendre.leggauss(p + 1)
    gx = 0.5 * (gx + 1.0)
    gw = 0.5 * gw
    cache = {}

    def cell_geom(leaf):
        l, i, j, k = leaf
        h = h0 / 2 ** l
        return h, np.array([lo + i * h, lo + j * h, lo + k * h])

    def coeffs(leaf):
        if leaf not in cache:
            h, c0 = cell_geom(leaf)
            pts = np.array([[c0[0] + h * xi[a], c0[1] + h * xi[b], c0[2] + h * xi[cc]]
                             for cc in range(p + 1) for b in range(p + 1) for a in range(p + 1)])
            cache[leaf] = _coulomb(pts, nuclei, h * wcube).reshape(p + 1, p + 1, p + 1)   # [c][b][a]
        return cache[leaf]

    def dn(leaf, X, d):
        """d/dx_d of the leaf's interpolant at the points X (m, 3)."""
        h, c0 = cell_geom(leaf)
        T = (X - c0[None, :]) / h
        Lx = gll.lagrange_matrix(xi, T[:, 0])
        Ly = gll.lagrange_matrix(xi, T[:, 1])
        Lz = gll.lagrange_matrix(xi, T[:, 2])
        D = gll.lagrange_deriv_matrix(xi, T[:, d]) / h
        M = [Lx, Ly, Lz]
        M[d] = D
        return np.einsum("cba,ma,mb,mc->m", coeffs(leaf), M[0], M[1], M[2])

    def face_points(c0, h, d, side):
        """Gauss points (m, 3) and weights (m,) of the face x_d = c0_d + side h."""
        o = [a for a in range(3) if a != d]
        U, W = np.meshgrid(gx, gx, indexing="ij")
        X = np.zeros((U.size, 3))
        X[:, d] = c0[d] + side * h
        X[:, o[0]] = c0[o[0]] + h * U.ravel()
        X[:, o[1]] = c0[o[1]] + h * W.ravel()
        wts = (gw[:, None] * gw[None, :]).ravel() * h * h
        return X, wts

    eta2 = {}
    for leaf in leafset:
        l, i, j, k = leaf
        h, c0 = cell_geom(leaf)
        if _contains_nucleus(c0, h, nuclei):
            eta2[leaf] = np.inf
            continue
        n = nc << l
        tot = 0.0
        for d in range(3):
            for side in (0, 1):
                nb = [i, j, k]
                nb[d] += 1 if side else -1
                if not (0 <= nb[d] < n):
                    continue
                f = _find_leaf(leafset, l, *nb)
                if f is not None:   # a leaf of the same or a coarser level covers the face
                    X, wts = face_points(c0, h, d, side)
                    J = dn(leaf, X, d) - dn(f, X, d)
                    tot += np.sum(wts * J * J)
                else:               # four finer leaves (2:1 balance), one quarter face each
                    hs = 0.5 * h
                    o = [a for a in range(3) if a != d]
                    for u in (0, 1):
                        for v in (0, 1):
                            ch = [2 * nb[0], 2 * nb[1], 2 * nb[2]]
                            ch[d] += 0 if side else 1
                            ch[o[0]] += u
                            ch[o[1]] += v
                            fine = (l + 1, ch[0], ch[1], ch[2])
                            cs = c0.copy()
                            cs[o[0]] += u * hs
                            cs[o[1]] += v * hs
                            X, wts = face_points(cs, hs, d, 0)
                            X[:, d] = c0[d] + side * h
                            J = dn(leaf, X, d) - dn(fine, X, d)
                            tot += np.sum(wts * J * J)
        eta2[leaf] = h / 24.0 * tot
    return eta2


def refine_leaves_kelly(nc, lo, h0, p, nuclei, theta, max_level):
    """Leaves after Kelly refinement (Sec. 3.1): starting from the uniform
    coarse cubes, every round splits each leaf with eta_K > theta (eta_K^2
    from `kelly_indicators`) whose level is below max_level (the smallest
    cell size; the largest is the coarse cube), then restores the 2:1 balance;
    rounds repeat until no leaf is split."""
    leaves = set(itertools.product([0], range(nc), range(nc), range(nc)))
    while True:
        eta2 = kelly_indicators(leaves, nc, lo, h0, p, nuclei)
        marked = [lf for lf in leaves if lf[0] < max_level and eta2[lf] > theta * theta]
        if not marked:
            return leaves
        for (l, i, j, k) in marked:
            leaves.remove((l, i, j, k))
            for a, b, d in itertools.product((0, 1), repeat=3):
                leaves.add((l + 1, 2 * i + a, 2 * j + b, 2 * k + d))
        leaves = balance_leaves(leaves, nc)


class Mesh:
    """Leaves, support points, masters, hanging constraints and the boundary.

    Attributes (all numpy):
      lev (ncell,), ijk (ncell, 3)     leaf level and integer position at its level
      h (ncell,), corner (ncell, 3)    side length and lower corner
      cell_pts (ncell, (p+1)^3)        support point of local node a + (p+1)(b + (p+1)c)
      X (nf, 3)                        coordinates of the support points
      hanging (nf,) bool               hanging-point flag
      master_of (nf,)                  master index of a point, -1 if hanging
      master_pts (N,)                  point index of each master
      C (nf, N) csr                    constraint matrix
      boundary (N,) bool               master lies on the box surface
      Xm (N, 3)                        master coordinates
    """

    def __init__(self, lo, hi, nc, p, nuclei, c=2.0, kelly=None):
        """kelly: None (the geometric rule) or (theta, max_level) for Kelly
        refinement on the Coulomb potential (`refine_leaves_kelly`)."""
        self.lo, self.hi, self.nc, self.p = float(lo), float(hi), int(nc), int(p)
        self.h0 = (self.hi - self.lo) / self.nc
        self.nuclei = [(np.asarray(R, dtype=np.float64), float(Z), int(L)) for (R, Z, L) in nuclei]
        self.c = float(c)
        self.xi, self.w = gll.gll_nodes_weights(self.p)
        if kelly is None:
            leaves = refine_leaves(self.nc, self.lo, self.h0, self.nuclei, self.c)
            leaves = balance_leaves(leaves, self.nc)
        else:
            leaves = refine_leaves_kelly(self.nc, self.lo, self.h0, self.p, self.nuclei, float(kelly[0]),
                                         int(kelly[1]))
        leaves = sorted(leaves)
        self.lev = np.array([t[0] for t in leaves], dtype=np.int64)
        self.ijk = np.array([t[1:] for t in leaves], dtype=np.int64)
        self.Lf = int(self.lev.max())
        self.h = self.h0 / 2.0 ** self.lev
        self.corner = self.lo + self.ijk * self.h[:, None]
        self._leafset = set(leaves)
        self._build_points()
        self._build_constraints()

    # ---------------------------------------------------------------- points
    def _node_keys(self):
        """Integer keys (ncell, (p+1)^3, 3) of every cell node, in units of h_finest / 2^KEY_BITS.

        A coordinate is (i + xi_a) cells of its level; keys of equal points are
        equal because rational nodes are exact and irrational nodes only meet
        the same node of the same column of cells.
        """
        p1 = self.p + 1
        scale = (2 ** (self.Lf - self.lev)).astype(np.int64) << KEY_BITS          # key units per cell
        off = np.rint(self.xi[None, :] * scale[:, None].astype(np.float64)).astype(np.int64)  # (ncell, p1)
        base = self.ijk * scale[:, None]                                        # (ncell, 3)
        kx = base[:, 0:1] + off                                                 # (ncell, p1)
        ky = base[:, 1:2] + off
        kz = base[:, 2:3] + off
        keys = np.empty((len(self.lev), p1 ** 3, 3), dtype=np.int64)
        for c_ in range(p1):
            for b in range(p1):
                for a in range(p1):
                    n = a + p1 * (b + p1 * c_)
                    keys[:, n, 0] = kx[:, a]
                    keys[:, n, 1] = ky[:, b]
                    keys[:, n, 2] = kz[:, c_]
        return keys

    def _build_points(self):
        keys = self._node_keys()
        ncell, nn, _ = keys.shape
        flat = keys.reshape(-1, 3)
        uniq, first, inv = np.unique(flat, axis=0, return_index=True, return_inverse=True)
        self.pkey = uniq
        self.cell_pts = inv.reshape(ncell, nn)
        # one (cell, local node) that carries each point, for exact local coordinates
        self.gen_cell = first // nn
        self.gen_node = first % nn
        unit = self.h0 / 2.0 ** self.Lf / 2.0 ** KEY_BITS
        self.X = self.lo + uniq.astype(np.float64) * unit
        self.nf = len(uniq)

    def containing_cells(self, pt):
        """All leaves whose closed box contains support point `pt` (by key arithmetic)."""
        K = self.pkey[pt]
        out = []
        for l in range(self.Lf + 1):
            s = (1 << (self.Lf - l)) << KEY_BITS
            n = self.nc << l
            cand = []
            for ax in range(3):
                q, r = divmod(int(K[ax]), s)
                opts = [q - 1, q] if r == 0 else [q]
                cand.append([v for v in opts if 0 <= v < n])
            for a in cand[0]:
                for b in cand[1]:
                    for d in cand[2]:
                        if (l, a, b, d) in self._leafset:
                            out.append((l, a, b, d))
        return out

    def _local_coords(self, pt, cell):
        """Coordinates of support point `pt` in the reference cube of `cell`.

        Computed from the leaf that carries the point as a node:
        t = (i_g 2^(l - l_g) - i) + xi_a 2^(l - l_g), where both terms are exact
        in floating point, so t is correctly rounded.
        """
        l, i, j, k = cell
        q = self.gen_cell[pt]
        n = self.gen_node[pt]
        p1 = self.p + 1
        loc = (n % p1, (n // p1) % p1, n // (p1 * p1))
        s = 2.0 ** (l - int(self.lev[q]))
        return np.array([(float(self.ijk[q, ax]) * s - float(c)) + self.xi[loc[ax]] * s
                         for ax, c in enumerate((i, j, k))])

    def _is_node(self, t):
        return all(np.min(np.abs(self.xi - t[ax])) < 1e-9 for ax in range(3))

    # ----------------------------------------------------------- constraints
    def _build_constraints(self):
        p1 = self.p + 1
        cell_index = {(int(self.lev[q]), *map(int, self.ijk[q])): q for q in range(len(self.lev))}
        # candidates: points on the boundary of some cell (interior nodes are never hanging)
        on_face = np.zeros(p1 ** 3, dtype=bool)
        for c_ in range(p1):
            for b in range(p1):
                for a in range(p1):
                    if a in (0, self.p) or b in (0, self.p) or c_ in (0, self.p):
                        on_face[a + p1 * (b + p1 * c_)] = True
        cand = np.unique(self.cell_pts[:, on_face])
        hanging = np.zeros(self.nf, dtype=bool)
        rows = {}
        for pt in cand:
            cells = self.containing_cells(pt)
            lmin = min(cl[0] for cl in cells)
            # Only the coarsest leaves around a point decide: a coarse node
            # inside a fine face is free, a fine node inside a coarse face is not.
            cell = next(cl for cl in cells if cl[0] == lmin)
            t = self._local_coords(pt, cell)
            if not self._is_node(t):
                hanging[pt] = True
                q = cell_index[cell]
                wts = np.kron(gll.lagrange_matrix(self.xi, t[2])[0],
                              np.kron(gll.lagrange_matrix(self.xi, t[1])[0],
                                      gll.lagrange_matrix(self.xi, t[0])[0]))
                nz = np.nonzero(wts)[0]
                rows[pt] = (self.cell_pts[q, nz], wts[nz])
        self.hanging = hanging
        self.master_pts = np.nonzero(~hanging)[0]
        self.N = len(self.master_pts)
        self.master_of = -np.ones(self.nf, dtype=np.int64)
        self.master_of[self.master_pts] = np.arange(self.N)
        r, cidx, v = [], [], []
        r.extend(self.master_pts.tolist())
        cidx.extend(range(self.N))
        v.extend([1.0] * self.N)
        for pt, (src, wts) in rows.items():
            m = self.master_of[src]
            if np.any(m < 0):
                raise RuntimeError("hanging point constrained by another hanging point")
            r.extend([pt] * len(m))
            cidx.extend(m.tolist())
            v.extend(wts.tolist())
        self.C = sp.csr_matrix((v, (r, cidx)), shape=(self.nf, self.N))
        self.Xm = self.X[self.master_pts]
        top = (self.nc << self.Lf) << KEY_BITS
        mk = self.pkey[self.master_pts]
        self.boundary = np.any((mk == 0) | (mk == top), axis=1)
        self.n_hanging = int(hanging.sum())

    def leaf_tuples(self):
        return sorted(zip(self.lev.tolist(), *[self.ijk[:, a].tolist() for a in range(3)]))
