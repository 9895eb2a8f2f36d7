"""Dense reference for the differentiation form: the one-electron limit of the
orbital step, its tangent and its adjoint (FP64).

With one orbital and one configuration the mean fields and the projector of
Eq. orb_eom vanish; the orbital obeys the length-gauge Schroedinger equation
with the one-body matrix of Sec. 3.1, integrated as in Sec. 3.2 with the
field frozen over each step.  On the interior masters (orbitals vanish on the
box surface), with M = diag(M_L):

    H~(E) = M^-1 H1~(E e),   Z~ = M^-1 F[e . r]    (so dH~/dE = Z~)
    phi_{k+1} = P_k phi_k,   P_k = expm(-i dt H~(E_k))
    d_k = <phi_k, O phi_k>_M = phi_k^H F[o] phi_k,  O = M^-1 F[o]

with o = e . r (the dipole) or o = e . f, f = -grad V the force of the
nuclei on the electron (the potential part of the Ehrenfest acceleration).

For a scalar objective with partial derivatives g_k = dJ/dd_k the chain rule
gives (<u, v>_M = u^H M v; A^+ = M^-1 A^H M the adjoint in that product):

    lam_K = g_K O phi_K,   lam_k = P_k^+ lam_{k+1} + g_k O phi_k
    dJ/dE_k = 2 Re <lam_{k+1}, L_k phi_k>_M,
    L_k = the Frechet derivative of expm at -i dt H~(E_k) in the direction -i dt Z~

and the tangent of a field perturbation v:
    dphi_{k+1} = P_k dphi_k + v_k L_k phi_k,   dd_k = 2 Re <O phi_k, dphi_k>_M.

Here every P_k and L_k is formed densely by scipy (expm, expm_frechet): slow
and only for tiny meshes, and a different route from the library's (which
propagates two stacked vectors by Krylov steps of a block operator).

Test infrastructure only (see the package docstring).
"""
import numpy as np
import scipy.linalg


class TDSE:
    """Dense one-electron propagator of an assembled mesh (see module docstring)."""

    def __init__(self, ops, e_dir=(0.0, 0.0, 1.0), observable="dipole"):
        self.ops = ops
        self.I = np.nonzero(ops.interior)[0]
        self.e = np.asarray(e_dir, dtype=np.float64)
        I = self.I
        self.m = ops.ML[I]
        self.H0 = ops.H1_matrix().toarray()[np.ix_(I, I)]
        Fr = ops.pointwise(ops.mesh.X @ self.e).toarray()[np.ix_(I, I)]
        self.Ht0 = self.H0 / self.m[:, None]          # M^-1 H1~(0)
        self.Zt = Fr / self.m[:, None]                # M^-1 F[e.r] = dH~/dE
        # the signal's matrix: F[e.r] (dipole) or F[e.f], f = -grad V (force)
        if observable == "dipole":
            self.F = Fr
        elif observable == "force":
            self.F = ops.pointwise(ops.nuclear_force(ops.mesh.X) @ self.e).toarray()[np.ix_(I, I)]
        else:
            raise ValueError("observable must be 'dipole' or 'force'")
        self.Ot = self.F / self.m[:, None]            # M^-1 F[observable]

    # ----------------------------------------------------------------- pieces
    def restrict(self, phi_full):
        return np.asarray(phi_full, dtype=np.complex128)[self.I]

    def Ht(self, E):
        return self.Ht0 + E * self.Zt

    def propagator(self, E, dt):
        return scipy.linalg.expm(-1j * dt * self.Ht(E))

    def dipole(self, phi):
        return float(np.real(np.conj(phi) @ (self.F @ phi)))

    def inner(self, u, v):
        return np.vdot(u, self.m * v)

    def adjoint_of(self, A):
        """A^+ = M^-1 A^H M."""
        return (A.conj().T * self.m[None, :]) / self.m[:, None]

    # ---------------------------------------------------------------- drivers
    def forward(self, phi0, E, dt):
        """Returns (d [K+1], phis [K+1][n_int])."""
        phis = [np.asarray(phi0, dtype=np.complex128)]
        for Ek in E:
            phis.append(self.propagator(Ek, dt) @ phis[-1])
        d = np.array([self.dipole(p) for p in phis])
        return d, phis

    def vjp(self, phi0, E, dt, g):
        """Returns (grad_E [K], lam_0) for the cotangent g [K+1] of the signal."""
        _, phis = self.forward(phi0, E, dt)
        K = len(E)
        lam = g[K] * (self.Ot @ phis[K])
        grad = np.zeros(K)
        for k in range(K - 1, -1, -1):
            P, L = scipy.linalg.expm_frechet(-1j * dt * self.Ht(E[k]), -1j * dt * self.Zt)
            grad[k] = 2.0 * np.real(self.inner(lam, L @ phis[k]))
            lam = self.adjoint_of(P) @ lam + g[k] * (self.Ot @ phis[k])
        return grad, lam

    def jvp(self, phi0, E, dt, v):
        """Returns (d [K+1], dd [K+1]) for the field perturbation v [K]."""
        phi = np.asarray(phi0, dtype=np.complex128)
        dphi = np.zeros_like(phi)
        d = [self.dipole(phi)]
        dd = [0.0]
        for k, Ek in enumerate(E):
            P, L = scipy.linalg.expm_frechet(-1j * dt * self.Ht(Ek), -1j * dt * self.Zt)
            dphi = P @ dphi + v[k] * (L @ phi)
            phi = P @ phi
            d.append(self.dipole(phi))
            dd.append(2.0 * np.real(self.inner(self.Ot @ phi, dphi)))
        return np.array(d), np.array(dd)
