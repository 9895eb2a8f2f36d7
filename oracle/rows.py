"""Selected rows of the assembled operators, computed cell by cell (FP64).

The operators are those of `fem` (Sec. 3.1): A = C^T A_f C with
A_f = sum_K P_K^T (h_K A_hat) P_K, F[f] = C^T diag(m_f o f) C, M_L = C^T m_f,
H1~ = 1/2 A + F[V + E . x].  For a mesh whose global matrices are too large to
assemble on the host, the row of master i follows from the support points p
with C_pi != 0 (i itself and the hanging points it constrains) and the cells
that carry them as nodes:

  (A x)_i     = sum_p C_pi sum_{(K, l): node l of K is p} h_K (A_hat (C x)|_K)_l
  (F[f] x)_i  = sum_p C_pi m_f,p f_p (C x)_p
  (M_L)_i     = sum_p C_pi m_f,p

and (M_L^-1 H1~ x)_i as `fem.Operators.h1_apply` forms it (x taken as 0 on the
box surface, rows of surface masters 0).  Only the rows asked for are formed.

Test infrastructure only (see the package docstring).
"""
import numpy as np

from . import fem


class RowOperators:
    """Row-wise evaluation of the operators of one mesh (see module docstring)."""

    def __init__(self, mesh):
        self.mesh = mesh
        p1 = mesh.p + 1
        nn = p1 ** 3
        self.A_hat, m_hat = fem.cell_matrices(mesh.p)
        self.m_f = np.bincount(mesh.cell_pts.ravel(), weights=(mesh.h[:, None] ** 3 * m_hat[None, :]).ravel(),
                               minlength=mesh.nf)
        self.CT = mesh.C.T.tocsr()
        self.ML = self.CT @ self.m_f
        self.interior = ~mesh.boundary
        # incidences (cell, local node) of every support point, grouped by point
        flat = mesh.cell_pts.ravel()
        order = np.argsort(flat, kind="stable")
        self.inc_ptr = np.searchsorted(flat[order], np.arange(mesh.nf + 1))
        self.inc_cell = order // nn
        self.inc_node = order % nn
        # the potential at the support points, exactly as the assembled operators take it
        self.V_f = fem.Operators.nuclear_potential(self, mesh.X)

    def _stiffness_row(self, i, xf):
        """(A x)_i from the full-point values xf = C x."""
        m = self.mesh
        a, b = self.CT.indptr[i], self.CT.indptr[i + 1]
        acc = np.zeros(xf.shape[1:], dtype=xf.dtype)
        for p, c in zip(self.CT.indices[a:b], self.CT.data[a:b]):
            for e in range(self.inc_ptr[p], self.inc_ptr[p + 1]):
                K = self.inc_cell[e]
                acc = acc + c * m.h[K] * (self.A_hat[self.inc_node[e]] @ xf[m.cell_pts[K]])
        return acc

    def stiffness_rows(self, rows, x):
        """(A x)[rows] (full Neumann stiffness), x: (N,) or (N, k)."""
        xf = self.mesh.C @ x
        return np.array([self._stiffness_row(i, xf) for i in rows])

    def h1_rows(self, rows, x, E=(0.0, 0.0, 0.0)):
        """(M_L^-1 H1~ x)[rows] with x taken as 0 on surface masters; surface rows are 0."""
        mask = self.interior.astype(np.float64)
        xm = x * (mask if x.ndim == 1 else mask[:, None])
        xf = self.mesh.C @ xm
        f = self.V_f + self.mesh.X @ np.asarray(E, dtype=np.float64)
        out = []
        for i in rows:
            if not self.interior[i]:
                out.append(np.zeros(xf.shape[1:], dtype=xf.dtype))
                continue
            a, b = self.CT.indptr[i], self.CT.indptr[i + 1]
            pts, c = self.CT.indices[a:b], self.CT.data[a:b]
            w = c * self.m_f[pts] * f[pts]
            pot = w @ xf[pts]
            out.append((0.5 * self._stiffness_row(i, xf) + pot) / self.ML[i])
        return np.array(out)
