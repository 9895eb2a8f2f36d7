"""Assembled finite-element operators over the master unknowns (FP64).

Sec. 3.1 defines the discretisation: the mass matrix M_kl = int b_k b_l, the
one-body matrix (H1)_kl = int b_k H1 b_l and every integral by GLL quadrature
on the cell nodes.  With collocated GLL quadrature the cell matrices of a cube
of side h are (1D factors on [0,1]; Khat the 1D stiffness, W = diag(w)):

  stiffness  A_K = h (Khat (x) W (x) W + W (x) Khat (x) W + W (x) W (x) Khat)
  mass       M_K = h^3 W (x) W (x) W      (diagonal)
  potential  F_K[f] = h^3 diag(w (x) w (x) w) diag(f at the nodes)

Assembly runs over the support points (A_f = sum_K P_K^T A_K P_K) and is then
constrained to the masters by C: A = C^T A_f C.  The mass used everywhere is
the lumped row-sum M_L = C^T m_f (m_f = assembled GLL weights); away from
hanging masters it equals the consistent GLL mass exactly.

The length-gauge one-body Hamiltonian is H1 = -1/2 Laplacian
- sum_a Z_a / |r - R_a| + E(t) . r, so its matrix is
H1~ = 1/2 A + F[V] + F[E . x], and orbitals vanish on the box surface.
In the velocity gauge of Sec. 2, H1 = -1/2 Laplacian - sum_a Z_a / |r - R_a|
- i A(t) . grad, the matrix is H1~ = 1/2 A + F[V] - i sum_d A_d G_d with G_d
the skew-symmetric form of int b_k d_d b_l: per cell h^2 (W (x) W (x) S) for
d = x (and its permutations), S = (Dw - Dw^T) / 2, Dw[i, j] = w_i L_j'(xi_i) =
int L_i L_j' (GLL quadrature is exact for this degree-(2p-1) product).  For
functions that vanish on the box surface the skew form equals the plain one
on a conforming mesh; on the hanging-node mesh it keeps -i A . G Hermitian,
which the plain form is not there (the lumped face quadratures of a coarse
face and its fine subfaces differ).

Exterior complex scaling (Sec. 4 absorbs the outgoing flux by ECS outside an
inner box, with the details left to the cited literature).  Reading taken
here: Cartesian scaling with a sharp onset at the faces of an inner box
|x_d| <= R_d, x_d -> +-R_d + e^{i theta} (x_d -+ R_d) outside, applied to the
kinetic energy; cells lie wholly inside or outside the box along each axis.
In the weak form a cell scaled along the axes f_d (eta_d = e^{i theta f_d},
J = prod_d eta_d) has the stiffness h sum_d (J / eta_d^2) (the d-th Kronecker
term) and the mass J h^3 W (x) W (x) W; with M_theta = C^T (J m_f) the
kinetic operator on nodal vectors is -1/2 Laplacian -> 1/2 M_theta^-1 A_theta.
The pointwise terms (nuclear potential, E . r, mean fields) keep their real
weights, and the orbital inner product stays <u, v> = u^H M_L v, so the
one-body matrix in that inner product is
H1~ = 1/2 diag(M_L / M_theta) A_theta + F[V + E . x]
(H1~ of the unscaled case when theta = 0).

Test infrastructure only (see the package docstring).
"""
import numpy as np
import scipy.sparse as sp

from . import gll

# Mean of 1/|r| over the unit cube centred at the origin: 3 ln(2 + sqrt 3) - pi/2.
CUBE_MEAN_INV_R = 3.0 * np.log(2.0 + np.sqrt(3.0)) - np.pi / 2.0


def cell_matrices(p):
    """(A_hat, m_hat): reference-cube stiffness (to be scaled by h) and mass diagonal (by h^3)."""
    xi, w = gll.gll_nodes_weights(p)
    K = gll.stiffness_1d(p)
    W = np.diag(w)
    A_hat = np.kron(W, np.kron(W, K)) + np.kron(W, np.kron(K, W)) + np.kron(K, np.kron(W, W))
    m_hat = np.kron(w, np.kron(w, w))
    return A_hat, m_hat


def gradient_matrices(p):
    """G_hat[d] (d = x, y, z): reference-cube matrices of the skew-symmetric
    form of int b_i d_d b_j (to be scaled by h^2); node index
    i = a + (p+1) (b + (p+1) c), a along x."""
    xi, w = gll.gll_nodes_weights(p)
    Dw = np.diag(w) @ gll.lagrange_deriv_matrix(xi, xi)
    S = 0.5 * (Dw - Dw.T)
    W = np.diag(w)
    return [np.kron(W, np.kron(W, S)), np.kron(W, np.kron(S, W)), np.kron(S, np.kron(W, W))]


def ecs_cell_flags(mesh, R, tol=1e-9):
    """(ncell, 3) 0/1: cell lies outside the inner box |x_d| <= R_d along axis d.
    ValueError when a face of the inner box cuts a cell."""
    R = np.asarray(R, dtype=np.float64)
    lo = mesh.corner
    hi = lo + mesh.h[:, None]
    inside = (lo >= -R - tol) & (hi <= R + tol)
    outside = (lo >= R - tol) | (hi <= -R + tol)
    if np.any(~(inside | outside)):
        raise ValueError("a face of the complex-scaling box cuts a cell")
    return outside.astype(np.int64)


class Operators:
    """Assembled sparse operators of one mesh (see module docstring)."""

    def __init__(self, mesh):
        self.mesh = mesh
        p1 = mesh.p + 1
        A_hat, m_hat = cell_matrices(mesh.p)
        nn = p1 ** 3
        ncell = len(mesh.lev)
        rows = np.repeat(mesh.cell_pts, nn, axis=1).ravel()
        cols = np.tile(mesh.cell_pts, (1, nn)).ravel()
        vals = (mesh.h[:, None, None] * A_hat[None, :, :]).reshape(ncell, -1).ravel()
        self.A_f = sp.csr_matrix((vals, (rows, cols)), shape=(mesh.nf, mesh.nf))
        self.m_f = np.bincount(mesh.cell_pts.ravel(),
                               weights=(mesh.h[:, None] ** 3 * m_hat[None, :]).ravel(),
                               minlength=mesh.nf)
        C = mesh.C
        self.C = C
        self.A = (C.T @ self.A_f @ C).tocsr()
        self.ML = C.T @ self.m_f
        self.interior = ~mesh.boundary
        self.V_f = self.nuclear_potential(mesh.X)

    # ----------------------------------------------------------- potentials
    def nuclear_potential(self, X):
        """V(x) = -sum_a Z_a / |x - R_a| at the support points X (nf, 3).

        At a support point that coincides with a nucleus the singular value is
        replaced by -Z c3 / s with s = m_f^(1/3) and c3 the mean of 1/|r| over
        a unit cube: the cell-averaged Coulomb value of a cube of the point's
        quadrature volume.
        """
        V = np.zeros(len(X))
        s = np.cbrt(self.m_f)
        for (R, Z, _L) in self.mesh.nuclei:
            d = np.linalg.norm(X - R[None, :], axis=1)
            on = d < 1e-10
            V[~on] -= Z / d[~on]
            V[on] -= Z * CUBE_MEAN_INV_R / s[on]
        return V

    def nuclear_force(self, X):
        """-grad V (nf, 3) at the support points X: -sum_a Z_a (x - R_a) / |x - R_a|^3,
        the force of the nuclei on an electron; 0 at a point on a nucleus (the
        cube-averaged force vanishes there by symmetry)."""
        F = np.zeros((len(X), 3))
        for (R, Z, _L) in self.mesh.nuclei:
            r = X - R[None, :]
            d = np.linalg.norm(r, axis=1)
            on = d < 1e-10
            F[~on] -= Z * r[~on] / d[~on, None] ** 3
        return F

    def pointwise(self, f):
        """F[f] = C^T diag(m_f o f) C for a function f given at the support points."""
        return (self.C.T @ sp.diags(self.m_f * f) @ self.C).tocsr()

    def gradient(self, d):
        """G_d = C^T (sum_K P_K^T h_K^2 Ghat_d P_K) C (assembled once per direction)."""
        if not hasattr(self, "_G"):
            self._G = [None, None, None]
        if self._G[d] is None:
            mesh = self.mesh
            nn = (mesh.p + 1) ** 3
            Gh = gradient_matrices(mesh.p)[d]
            rows = np.repeat(mesh.cell_pts, nn, axis=1).ravel()
            cols = np.tile(mesh.cell_pts, (1, nn)).ravel()
            vals = (mesh.h[:, None, None] ** 2 * Gh[None, :, :]).reshape(len(mesh.lev), -1).ravel()
            Gf = sp.csr_matrix((vals, (rows, cols)), shape=(mesh.nf, mesh.nf))
            self._G[d] = (self.C.T @ Gf @ self.C).tocsr()
        return self._G[d]

    def set_ecs(self, theta, R):
        """Exterior complex scaling of the kinetic energy outside |x_d| <= R_d
        by the angle theta (module docstring); theta = 0 removes it."""
        self.ecs = None
        if theta == 0.0:
            return
        mesh = self.mesh
        f = ecs_cell_flags(mesh, R)
        eta = np.exp(1j * theta)
        J = eta ** f.sum(axis=1)
        s = J[:, None] / eta ** (2 * f)            # (ncell, 3): J / eta_d^2
        K = gll.stiffness_1d(mesh.p)
        W = np.diag(mesh.w)
        Ad = [np.kron(W, np.kron(W, K)), np.kron(W, np.kron(K, W)), np.kron(K, np.kron(W, W))]
        nn = (mesh.p + 1) ** 3
        ncell = len(mesh.lev)
        vals = mesh.h[:, None, None] * (s[:, 0, None, None] * Ad[0][None] + s[:, 1, None, None] * Ad[1][None]
                                        + s[:, 2, None, None] * Ad[2][None])
        rows = np.repeat(mesh.cell_pts, nn, axis=1).ravel()
        cols = np.tile(mesh.cell_pts, (1, nn)).ravel()
        Af = sp.csr_matrix((vals.reshape(ncell, -1).ravel(), (rows, cols)), shape=(mesh.nf, mesh.nf))
        self.A_theta = (self.C.T @ Af @ self.C).tocsr()
        _, m_hat = cell_matrices(mesh.p)
        wts = (J[:, None] * mesh.h[:, None] ** 3 * m_hat[None, :]).ravel()
        pts = mesh.cell_pts.ravel()
        m_theta_f = (np.bincount(pts, weights=wts.real, minlength=mesh.nf)
                     + 1j * np.bincount(pts, weights=wts.imag, minlength=mesh.nf))
        self.M_theta = self.C.T @ m_theta_f
        self.rho = self.ML / self.M_theta
        self.ecs = (float(theta), tuple(float(r) for r in R), f)

    def H1_matrix(self, E=(0.0, 0.0, 0.0), A=None):
        """H1~ = 1/2 A + F[V + E . x] over all masters (boundary rows/cols kept);
        with a vector potential A (velocity gauge, Sec. 2) the term
        -i sum_d A_d G_d is added (complex matrix); with complex scaling
        (set_ecs) the kinetic part is 1/2 diag(M_L / M_theta) A_theta."""
        E = np.asarray(E, dtype=np.float64)
        f = self.V_f + self.mesh.X @ E
        if getattr(self, "ecs", None) is not None:
            if A is not None and np.any(np.asarray(A) != 0.0):
                raise ValueError("complex scaling is built for the length gauge")
            return (0.5 * sp.diags(self.rho) @ self.A_theta + self.pointwise(f)).tocsr()
        H = 0.5 * self.A + self.pointwise(f)
        if A is not None and np.any(np.asarray(A) != 0.0):
            for d in range(3):
                if A[d] != 0.0:
                    H = H - 1j * A[d] * self.gradient(d)
        return H.tocsr()

    def h1_apply(self, x, E=(0.0, 0.0, 0.0), A=None):
        """y = M_L^{-1} H1~ x on interior masters; boundary entries of x are taken as 0
        and boundary entries of y are 0 (orbitals vanish on the box surface).

        x: (N,) or (N, nvec), real or complex.  A: vector potential (velocity gauge).
        """
        H = self.H1_matrix(E, A)
        mask = self.interior.astype(np.float64)
        xm = x * (mask if x.ndim == 1 else mask[:, None])
        y = H @ xm
        scale = mask / self.ML
        return y * (scale if y.ndim == 1 else scale[:, None])

    def stiffness_apply(self, x):
        """y = A x (full Neumann stiffness over all masters)."""
        return self.A @ x

    def full_values(self, x):
        """Values at all support points of the FE function with master coefficients x (C x)."""
        return self.C @ x
