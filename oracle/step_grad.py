"""Gradient of a signal of the full MCTDHF step with respect to the field:
the differentiation form beyond the one-electron limit.  Tiny meshes only.

The step of `mctdhf.MCTDHF.step` (Sec. 2, Sec. 3.2) is restated as dense maps
of the interior orbital coefficients phi (N_I x n) and the CI vector c, in
PyTorch (CPU, complex128), so that torch.autograd forms dJ/dE_k:

  rho_rs  = conj(C_I phi_r) o (C_I phi_s)          pair densities at the support points
  W_rs    = P rho_rs                               Poisson with multipole surface data
            (Eq. mean-field), P = [A_II^-1 (b - A_IB B); B] with b = 4 pi C^T diag(m_f)
            and B the multipole map to the surface masters (the oracle's own
            right-hand side and boundary routine applied to unit densities)
  h_pq    = phi_p^H H1~(E) phi_q,   H1~(E) = H1~(0) + E F[e . x]
  (pq|rs) = sum_f m_f conj(C_I phi_p) (C_I phi_q) (C W_rs)
  H_CI    = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps)
  c'      = exp(-i dt H_CI) c
  gamma_pq = c^H E_pq c,   Gamma_pqrs = c^H (E_pq E_rs - delta_qr E_ps) c
  U_pq    = sum_o (gamma^-1)_po sum_rs Gamma_oqrs W_rs
  phi'    = exp(-i dt G) phi,   (G v)_p = Q M^-1 [ H1~(E) v_p + C_I^T diag(m_f o C U_pq) C_I v_q ]
            summed over q, Q y = y - sum_j phi_j (phi_j^H M y)
  d       = Re sum_pq gamma_pq phi_p^H F[e . x] phi_q      (the signal at t, before the step)

with the field E e frozen over each step at its left point.  The orbital step
is the exact exponential of G (the library's Krylov step reaches it within its
error estimate).  J = sum_k g_k d_k over the signal at t_0 .. t_K; the
gradient dJ/dE is formed by reverse-mode differentiation, the tangent
dd = (dd_k/dE) v along a field perturbation v by its forward counterpart.

Test infrastructure only (see the package docstring).
"""
import numpy as np
import torch


class DenseMCTDHF:
    """Dense differentiable MCTDHF step on the interior masters of a tiny mesh.

    sim: an `mctdhf.MCTDHF` of the same mesh (its operators, Poisson solver
    and CI space are read, not changed).
    """

    def __init__(self, sim, e_dir=(0.0, 0.0, 1.0)):
        ops, m, ps, ci = sim.ops, sim.mesh, sim.ps, sim.ci
        self.n = sim.n
        self.I = np.nonzero(~m.boundary)[0]
        I = self.I
        e = np.asarray(e_dir, dtype=np.float64)

        def t(a):
            return torch.from_numpy(np.ascontiguousarray(a))

        self.ML = t(ops.ML[I]).to(torch.complex128)
        self.H0 = t(ops.H1_matrix((0.0, 0.0, 0.0)).toarray()[np.ix_(I, I)]).to(torch.complex128)
        Fe = sum(e[d] * ops.pointwise(m.X[:, d]).toarray()[np.ix_(I, I)] for d in range(3))
        self.Fe = t(Fe).to(torch.complex128)
        Cfull = ops.C.toarray()
        self.C = t(Cfull).to(torch.complex128)
        self.CI = t(Cfull[:, I]).to(torch.complex128)
        self.mf = t(ops.m_f).to(torch.complex128)
        # the Poisson solution operator on real densities, applied to complex ones
        # column by column (it is real and linear)
        b, g = ps.rhs_and_bc(np.eye(m.nf))
        P = np.zeros((m.N, m.nf))
        P[ps.B] = g
        P[ps.I] = np.linalg.solve(ps.A_II.toarray(), b[ps.I] - ps.A_IB @ g)
        self.P = t(P).to(torch.complex128)
        n, D = self.n, ci.dim
        E1 = np.zeros((n, n, D, D))
        E2 = np.zeros((n, n, n, n, D, D))
        for p in range(n):
            for q in range(n):
                E1[p, q] = ci.E[p][q].toarray()
        for p in range(n):
            for q in range(n):
                for r in range(n):
                    for s in range(n):
                        M = E1[p, q] @ E1[r, s]
                        if q == r:
                            M = M - E1[p, s]
                        E2[p, q, r, s] = M
        self.E1 = t(E1).to(torch.complex128)
        self.E2 = t(E2).to(torch.complex128)

    def restrict(self, phi_full):
        return torch.from_numpy(np.ascontiguousarray(np.asarray(phi_full, dtype=np.complex128)[self.I]))

    def signal(self, phi, c):
        """d = Re sum_pq gamma_pq phi_p^H F[e.x] phi_q."""
        g1 = torch.einsum("i,pqij,j->pq", c.conj(), self.E1, c)
        Z = phi.conj().T @ (self.Fe @ phi)
        return torch.real(torch.sum(g1 * Z))

    def step(self, phi, c, E, dt):
        """(phi', c') of one step with the field amplitude E (real scalar tensor) along e."""
        n, NI = self.n, phi.shape[0]
        H1 = self.H0 + E * self.Fe
        pf = self.CI @ phi                                          # (nf, n)
        rho = pf.conj()[:, :, None] * pf[:, None, :]                # rho[f, r, s]
        W = torch.einsum("Nf,frs->rsN", self.P, rho)               # (n, n, N)
        Wf = torch.einsum("fN,rsN->rsf", self.C, W)                # (n, n, nf)
        h = phi.conj().T @ (H1 @ phi)
        dens = self.mf[:, None, None] * rho                         # m_f conj(phi_p) phi_q
        eri = torch.einsum("fpq,rsf->pqrs", dens, Wf)
        Hci = torch.einsum("pq,pqij->ij", h, self.E1) + 0.5 * torch.einsum("pqrs,pqrsij->ij", eri, self.E2)
        Hci = 0.5 * (Hci + Hci.conj().T)
        c_new = torch.linalg.matrix_exp(-1j * dt * Hci) @ c
        g1 = torch.einsum("i,pqij,j->pq", c.conj(), self.E1, c)
        g2 = torch.einsum("i,pqrsij,j->pqrs", c.conj(), self.E2, c)
        U = torch.einsum("po,oqrs,rsN->pqN", torch.linalg.inv(g1), g2, W)
        Uf = torch.einsum("fN,pqN->pqf", self.C, U)
        blocks = []
        for p in range(n):
            row = []
            for q in range(n):
                B = self.CI.T @ ((self.mf * Uf[p, q])[:, None] * self.CI)
                if p == q:
                    B = B + H1
                row.append(B / self.ML[:, None])
            blocks.append(torch.cat(row, dim=1))
        Y = torch.cat(blocks, dim=0)                                # M^-1 [H1 (x) I + mean field]
        Q = torch.eye(NI, dtype=torch.complex128) - phi @ (phi.conj().T * self.ML[None, :])
        G = torch.block_diag(*([Q] * n)) @ Y
        v = phi.T.reshape(-1)                                       # orbital-major stacking
        phi_new = (torch.linalg.matrix_exp(-1j * dt * G) @ v).reshape(n, NI).T
        return phi_new, c_new

    def signals(self, phi0, c0, E, dt):
        """d_0 .. d_K for the K field amplitudes E (real tensor)."""
        phi, c = phi0, c0
        d = [self.signal(phi, c)]
        for k in range(E.shape[0]):
            phi, c = self.step(phi, c, E[k], dt)
            d.append(self.signal(phi, c))
        return torch.stack(d)

    def gradient(self, phi0, c0, E, dt, g):
        """(J, dJ/dE) for J = sum_k g_k d_k (numpy in, numpy out)."""
        Et = torch.tensor(np.asarray(E, dtype=np.float64), requires_grad=True)
        d = self.signals(phi0, c0, Et, dt)
        J = torch.sum(torch.from_numpy(np.asarray(g, dtype=np.float64)) * d)
        J.backward()
        return float(J.detach()), Et.grad.numpy().copy()

    def tangent(self, phi0, c0, E, dt, v):
        """(d [K+1], dd [K+1]): the signal and its derivative along the field
        perturbation v [K] (numpy in, numpy out)."""
        Et = torch.tensor(np.asarray(E, dtype=np.float64))
        vt = torch.tensor(np.asarray(v, dtype=np.float64))
        d, dd = torch.autograd.functional.jvp(lambda x: self.signals(phi0, c0, x, dt), Et, vt)
        return d.detach().numpy().copy(), dd.detach().numpy().copy()
