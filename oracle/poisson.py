"""Mean-field potentials by the Poisson equation (Sec. 3.1, Eq. mean-field).

W^r_s(x) = int phi_r*(x') phi_s(x') / |x - x'| dx' is obtained from
Delta W = -4 pi phi_r* phi_s with Dirichlet data on the box surface equal to
the direct integral.  In weak form with GLL quadrature:

    A W = 4 pi C^T (m_f o rho_f),   rho_f = conj(C phi_r) o (C phi_s),

solved on the interior masters with W fixed to g on the surface masters:
A_II W_I = b_I - A_IB g_B.  The surface data g is the direct integral written
as a multipole expansion about the box centre (reading of the paper, which
leaves the evaluation method open), truncated at l <= LMAX:

    g(x) = sum_lm 4 pi / (2l + 1) q_lm Y_lm(x^) / r^(l+1),
    q_lm = sum_f m_f rho_f r_f^l Y_lm(x_f^),

with real orthonormal spherical harmonics Y_lm.  Complex pair densities are
solved as two real right-hand sides (real and imaginary parts).

Test infrastructure only (see the package docstring).
"""
import math

import numpy as np
import scipy.sparse.linalg as sla
from scipy import special

LMAX = 12


def real_sph_harm(l, m, theta, phi):
    """Real orthonormal Y_lm(theta, phi) from associated Legendre functions.

    m > 0: sqrt2 N P_l^m(cos t) cos(m p);  m < 0: sqrt2 N P_l^|m| sin(|m| p);
    m = 0: N P_l(cos t);  N = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!).
    """
    am = abs(m)
    N = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    P = special.lpmv(am, l, np.cos(theta))
    if m == 0:
        return N * P
    if m > 0:
        return math.sqrt(2.0) * N * P * np.cos(am * phi)
    return math.sqrt(2.0) * N * P * np.sin(am * phi)


def _spherical(X, center):
    d = X - center[None, :]
    r = np.linalg.norm(d, axis=1)
    theta = np.arccos(np.clip(d[:, 2] / np.where(r > 0, r, 1.0), -1.0, 1.0))
    phi = np.arctan2(d[:, 1], d[:, 0])
    return r, theta, phi


def multipole_moments(X, weights, rho, center, lmax=LMAX):
    """q[l][m + l] = sum_f weights_f rho_f r_f^l Y_lm(x_f^) for real rho (nf,) or (nf, k)."""
    r, th, ph = _spherical(X, center)
    rho2 = rho.reshape(len(X), -1)
    q = {}
    for l in range(lmax + 1):
        rl = r ** l
        for m in range(-l, l + 1):
            q[(l, m)] = (weights * rl * real_sph_harm(l, m, th, ph)) @ rho2
    return q


def multipole_potential(q, Xb, center, lmax=LMAX):
    """g(x) = sum_lm 4 pi/(2l+1) q_lm Y_lm(x^) / r^(l+1) at points Xb (nb, 3)."""
    r, th, ph = _spherical(Xb, center)
    k = next(iter(q.values())).shape[0]
    g = np.zeros((len(Xb), k))
    for l in range(lmax + 1):
        fac = 4.0 * math.pi / (2 * l + 1) / r ** (l + 1)
        for m in range(-l, l + 1):
            g += np.outer(fac * real_sph_harm(l, m, th, ph), q[(l, m)])
    return g


def direct_potential(X, weights, rho, Xb):
    """The literal direct integral by the same quadrature: sum_f w_f rho_f / |x_b - x_f|."""
    out = np.zeros((len(Xb),) + rho.shape[1:])
    for b in range(len(Xb)):
        d = np.linalg.norm(X - Xb[b][None, :], axis=1)
        far = d > 0.0
        if np.any(rho[~far] != 0):
            raise ValueError("direct potential requested at a point carrying charge")
        out[b] = (weights[far] / d[far]) @ rho[far]
    return out


class PoissonSolver:
    """Dirichlet Poisson solves on one mesh (see module docstring)."""

    def __init__(self, ops, lmax=LMAX):
        self.ops = ops
        self.mesh = ops.mesh
        self.lmax = lmax
        m = self.mesh
        self.center = np.full(3, 0.5 * (m.lo + m.hi))
        self.I = np.nonzero(~m.boundary)[0]
        self.B = np.nonzero(m.boundary)[0]
        A = ops.A
        self.A_II = A[self.I][:, self.I].tocsr()
        self.A_IB = A[self.I][:, self.B].tocsr()
        self.Xb = m.Xm[self.B]
        self._lu = None

    def rhs_and_bc(self, rho_f):
        """(b, g_B) for real densities rho_f at the support points, shape (nf, k)."""
        ops = self.ops
        rho_f = rho_f.reshape(self.mesh.nf, -1)
        b = 4.0 * np.pi * (ops.C.T @ (ops.m_f[:, None] * rho_f))
        q = multipole_moments(self.mesh.X, ops.m_f, rho_f, self.center, self.lmax)
        g = multipole_potential(q, self.Xb, self.center, self.lmax)
        return b, g

    def solve(self, rho_f, method="direct", rtol=1e-12, x0=None):
        """W (N, k) with W_B = g and A_II W_I = b_I - A_IB g_B.

        method: "direct" (sparse LU) or "cg" (Jacobi-preconditioned CG to
        ||r|| <= rtol ||b_eff||).
        """
        b, g = self.rhs_and_bc(rho_f)
        k = b.shape[1]
        rhs = b[self.I] - self.A_IB @ g
        W = np.zeros((self.mesh.N, k))
        W[self.B] = g
        if method == "direct":
            if self._lu is None:
                self._lu = sla.splu(self.A_II.tocsc())
            W[self.I] = self._lu.solve(rhs)
        else:
            d = self.A_II.diagonal()
            Minv = sla.LinearOperator(self.A_II.shape, matvec=lambda v: v / d)
            for j in range(k):
                xs = None if x0 is None else x0[self.I, j]
                sol, info = sla.cg(self.A_II, rhs[:, j], x0=xs, rtol=rtol, atol=0.0, M=Minv,
                                   maxiter=100000)
                if info != 0:
                    raise RuntimeError("oracle CG did not converge")
                W[self.I, j] = sol
        return W

    def residual(self, W, rho_f):
        """||b_I - A_II W_I - A_IB W_B|| / ||b_I - A_IB g_B|| per column (backward error)."""
        b, g = self.rhs_and_bc(rho_f)
        rhs = b[self.I] - self.A_IB @ g
        r = b[self.I] - self.A_II @ W[self.I] - self.A_IB @ W[self.B]
        return np.linalg.norm(r, axis=0) / np.linalg.norm(rhs, axis=0)


def pair_densities(ops, phi):
    """Real right-hand-side densities of all pairs r <= s at the support points.

    phi: (N, n) complex master coefficients.  Returns (rho (nf, n*n) real, pairs)
    with pairs[j] = (r, s, part) listing each column: part 0 = real part of
    conj(phi_r) phi_s, part 1 = imaginary part (only for r < s).  The column
    order is: diagonal pairs first (r = s), then r < s as (re, im).
    """
    pf = ops.C @ phi
    n = phi.shape[1]
    cols, pairs = [], []
    for r in range(n):
        cols.append(np.abs(pf[:, r]) ** 2)
        pairs.append((r, r, 0))
    for r in range(n):
        for s in range(r + 1, n):
            z = np.conj(pf[:, r]) * pf[:, s]
            cols.append(z.real)
            pairs.append((r, s, 0))
            cols.append(z.imag)
            pairs.append((r, s, 1))
    return np.stack(cols, axis=1), pairs


def assemble_pair_potentials(Wcols, pairs, n):
    """Complex W[r][s] (N,) from the real solution columns; W_sr = conj(W_rs)."""
    N = Wcols.shape[0]
    W = np.zeros((n, n, N), dtype=np.complex128)
    for j, (r, s, part) in enumerate(pairs):
        if part == 0:
            W[r, s] += Wcols[:, j]
        else:
            W[r, s] += 1j * Wcols[:, j]
    for r in range(n):
        for s in range(r + 1, n):
            W[s, r] = np.conj(W[r, s])
    return W
