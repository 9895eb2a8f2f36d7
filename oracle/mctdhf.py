"""One MCTDHF time step on the FE mesh (Sec. 2 and Sec. 3.2).

Notation (see ``ci``): gamma, Gamma are the spin-summed RDMs, W[r][s] the
pair mean fields of Eq. mean-field, h_pq = phi_p^H H1~ phi_q and
(pq|rs) = sum_f m_f conj(phi_p) phi_q W_rs at the support points.

Orbital equation (Eq. orb_eom with X = 0, discretised as Eq.
discretized_eom with the lumped mass; orbitals are nodal coefficients):

  i dphi_p/dt = Q [ M_L^-1 H1~ phi_p + M_L^-1 C^T diag(m_f) sum_q U_pq o (C phi_q) ],
  U_pq = sum_o (gamma^-1)_po sum_rs Gamma_oqrs W_rs,
  Q y = y - sum_j phi_j (phi_j^H M_L y).

The packed operator G of Eq. packed_orb_eom freezes phi, gamma, Gamma, W and
the field at t, so phi(t+dt) = exp(-i G dt) phi(t) by the short-iterative
Arnoldi scheme (Sec. 3.2).  The CI vector is advanced with the exact
exponential of the frozen CI Hamiltonian (Eq. ci_eom with X = 0), from the
same time-t quantities.

Test infrastructure only (see the package docstring).
"""
import numpy as np
import scipy.linalg

from . import ci as ci_mod
from . import krylov, poisson


class MCTDHF:
    def __init__(self, ops, n_orb, n_alpha, n_beta, poisson_method="direct", poisson_rtol=1e-12):
        self.ops = ops
        self.mesh = ops.mesh
        self.n = n_orb
        self.ci = ci_mod.CISpace(n_orb, n_alpha, n_beta)
        self.ps = poisson.PoissonSolver(ops)
        self.poisson_method = poisson_method
        self.poisson_rtol = poisson_rtol
        self.interior = (~self.mesh.boundary).astype(np.float64)
        self.gauge = "length"

    # --------------------------------------------------------------- pieces
    def h1(self, E):
        """H1~ at the field argument E: the field E(t) in the length gauge, the
        vector potential A(t) in the velocity gauge (Sec. 2)."""
        if getattr(self, "gauge", "length") == "velocity":
            return self.ops.H1_matrix((0.0, 0.0, 0.0), A=E)
        return self.ops.H1_matrix(E)

    def inner(self, u, v):
        """<u, v> = sum_p u_p^H M_L v_p for stacked orbitals (N, n)."""
        return np.sum(np.conj(u) * (self.ops.ML[:, None] * v))

    def mean_fields(self, phi):
        """W[r][s] (N,) for all pairs (Eq. mean-field via the Poisson equation)."""
        rho, pairs = poisson.pair_densities(self.ops, phi)
        Wc = self.ps.solve(rho, method=self.poisson_method, rtol=self.poisson_rtol)
        return poisson.assemble_pair_potentials(Wc, pairs, self.n), Wc

    def integrals(self, phi, W, E):
        """h_pq = phi_p^H H1~(E) phi_q and (pq|rs) = sum_f m_f conj(phi_p) phi_q W_rs."""
        H1 = self.h1(E)
        pm = phi * self.interior[:, None]
        h = np.conj(pm).T @ (H1 @ pm)
        pf = self.ops.C @ pm
        Wf = np.stack([[self.ops.C @ W[r, s] for s in range(self.n)] for r in range(self.n)])
        n = self.n
        eri = np.zeros((n, n, n, n), dtype=np.complex128)
        for p in range(n):
            for q in range(n):
                d = self.ops.m_f * np.conj(pf[:, p]) * pf[:, q]
                for r in range(n):
                    for s in range(n):
                        eri[p, q, r, s] = np.sum(d * Wf[r, s])
        return h, eri

    def mean_field_operator(self, g1, g2, W):
        """U[p][q] (N,) = sum_o (gamma^-1)_po sum_rs Gamma_oqrs W_rs."""
        n = self.n
        ginv = np.linalg.inv(g1)
        Gam = np.einsum("po,oqrs->pqrs", ginv, g2)
        return np.einsum("pqrs,rsk->pqk", Gam, W)

    def G_apply(self, v, phi, U, E):
        """(G v)_p = Q [ M_L^-1 (H1~ v_p + C^T diag(m_f) sum_q (C U_pq) o (C v_q)) ] (interior)."""
        ops = self.ops
        n = self.n
        H1 = self.h1(E)
        msk = self.interior[:, None]
        vm = v * msk
        z = H1 @ vm
        vf = ops.C @ vm
        for p in range(n):
            acc = np.zeros(ops.mesh.nf, dtype=np.complex128)
            for q in range(n):
                acc += (ops.C @ U[p, q]) * vf[:, q]
            z[:, p] += ops.C.T @ (ops.m_f * acc)
        y = z * msk / ops.ML[:, None]
        S = np.conj(phi).T @ (ops.ML[:, None] * y)     # S[j, p] = phi_j^H M_L y_p
        return y - phi @ S

    # ----------------------------------------------------------------- step
    def step(self, phi, C, E, dt, m, krylov_tol=0.0, krylov_adaptive=0):
        """One step t -> t + dt.  Returns (phi_new, C_new, info dict).

        krylov_tol <= 0: the orbitals take one Krylov step of dimension m over
        dt.  krylov_tol > 0: the error-controlled substeps of
        ``krylov.arnoldi_propagate`` (estimate <= krylov_tol * beta per substep,
        Sec. 3.2); info then carries the substep count, the summed estimates
        and the decisions' smallest margin to the threshold.  krylov_adaptive > 0
        (with krylov_tol > 0): the rule of Sec. 3.2, ``krylov.arnoldi_adaptive``
        with that many equal steps and dimensions up to m."""
        W, Wc = self.mean_fields(phi)
        h, eri = self.integrals(phi, W, E)
        Hci = self.ci.hamiltonian(h, eri)
        g1 = self.ci.rdm1(C)
        g2 = self.ci.rdm2(C)
        if getattr(self.ops, "ecs", None) is not None:
            # complex scaling: h_pq, and so H_CI, is not Hermitian
            C_new = scipy.linalg.expm(-1j * dt * Hci) @ C
        else:
            evals, evecs = np.linalg.eigh(0.5 * (Hci + Hci.conj().T))
            C_new = evecs @ (np.exp(-1j * dt * evals) * (evecs.conj().T @ C))
        U = self.mean_field_operator(g1, g2, W)
        apply_G = lambda v: self.G_apply(v, phi, U, E)   # noqa: E731
        substeps, margin, Hk, m_used, brk = 1, np.inf, None, m, False
        dims = None
        if krylov_tol > 0.0 and krylov_adaptive > 0:
            phi_new, err, pinfo = krylov.arnoldi_adaptive(apply_G, phi, self.inner, m, dt, krylov_tol,
                                                          substeps=krylov_adaptive)
            margin, dims, substeps = pinfo["margin"], pinfo["dims"], krylov_adaptive
        elif krylov_tol > 0.0:
            phi_new, err, substeps, pinfo = krylov.arnoldi_propagate(apply_G, phi, self.inner, m, dt, krylov_tol,
                                                                     return_info=True)
            margin = pinfo["margin"]
        else:
            phi_new, err, Hk, m_used, brk = krylov.arnoldi_expm(apply_G, phi, self.inner, m, dt)
        energy = np.real(np.sum(h * g1) + 0.5 * np.einsum("pqrs,pqrs->", eri, g2))
        info = dict(W=W, Wcols=Wc, h=h, eri=eri, Hci=Hci, gamma=g1, Gamma=g2, U=U,
                    arnoldi_err=err, H_krylov=Hk, m_used=m_used, breakdown=brk, energy=energy,
                    krylov_substeps=substeps, krylov_margin=margin, krylov_dims=dims,
                    dipole=self.dipole(phi, C))
        return phi_new, C_new, info

    def step_imaginary(self, phi, C, dtau, m, krylov_tol=0.0, E=(0.0, 0.0, 0.0)):
        """One imaginary-time step tau -> tau + dtau toward the ground state
        (Sec. 4 prepares the initial state by imaginary-time propagation; the
        paper gives no scheme, reading 20).  The real-time step with t = -i tau:
        the same frozen quantities, C <- exp(-dtau H_CI) C normalised, and
        phi <- exp(-dtau G) phi by the Arnoldi process (one Krylov step, or the
        error-controlled substeps when krylov_tol > 0), followed by Loewdin
        orthonormalisation phi <- phi S^-1/2, S = phi^H M_L phi (the step leaves
        S - I of second order in dtau).  Returns (phi_new, C_new, info); the
        energy is that of the input state."""
        W, Wc = self.mean_fields(phi)
        h, eri = self.integrals(phi, W, E)
        Hci = self.ci.hamiltonian(h, eri)
        g1 = self.ci.rdm1(C)
        g2 = self.ci.rdm2(C)
        evals, evecs = np.linalg.eigh(0.5 * (Hci + Hci.conj().T))
        C_new = evecs @ (np.exp(-dtau * (evals - evals[0])) * (evecs.conj().T @ C))
        C_new = C_new / np.linalg.norm(C_new)
        U = self.mean_field_operator(g1, g2, W)
        apply_G = lambda v: self.G_apply(v, phi, U, E)   # noqa: E731
        if krylov_tol > 0.0:
            phi_new, err, substeps = krylov.arnoldi_propagate(apply_G, phi, self.inner, m, dtau, krylov_tol,
                                                              imaginary=True)
        else:
            phi_new, err, _, _, _ = krylov.arnoldi_expm(apply_G, phi, self.inner, m, dtau, imaginary=True)
            substeps = 1
        S = np.conj(phi_new).T @ (self.ops.ML[:, None] * phi_new)
        lam, V = np.linalg.eigh(0.5 * (S + S.conj().T))
        phi_new = phi_new @ (V @ np.diag(lam ** -0.5) @ V.conj().T)
        energy = np.real(np.sum(h * g1) + 0.5 * np.einsum("pqrs,pqrs->", eri, g2))
        return phi_new, C_new, dict(energy=energy, arnoldi_err=err, krylov_substeps=substeps,
                                    overlap_drift=np.abs(S - np.eye(self.n)).max())

    def dipole(self, phi, C):
        """<sum_i r_i> (3,): sum_pq gamma_pq phi_p^H F[x_d] phi_q, the one-body
        expectation of the summed electron positions (the length-gauge field term
        of Sec. 2 is E . r per electron, so this is dE_total/dE; the dipole moment
        is its negative)."""
        g1 = self.ci.rdm1(C)
        pm = phi * self.interior[:, None]
        out = np.zeros(3)
        for d in range(3):
            F = self.ops.pointwise(self.mesh.X[:, d])
            Z = np.conj(pm).T @ (F @ pm)
            out[d] = np.real(np.sum(Z * g1))
        return out

    def energy(self, phi, C, E=(0.0, 0.0, 0.0)):
        """E = sum_pq h_pq gamma_pq + 1/2 sum (pq|rs) Gamma_pqrs (electronic, no nuclear repulsion)."""
        W, _ = self.mean_fields(phi)
        h, eri = self.integrals(phi, W, E)
        g1 = self.ci.rdm1(C)
        g2 = self.ci.rdm2(C)
        return np.real(np.sum(h * g1) + 0.5 * np.einsum("pqrs,pqrs->", eri, g2))
