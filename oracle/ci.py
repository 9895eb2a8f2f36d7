"""Determinant space, spin-summed excitation operators, RDMs and the CI
Hamiltonian of MCTDHF (Sec. 2).

The MCTDHF wave function is a combination of all Slater determinants of n
spatial orbitals (Sec. 2).  A determinant is a pair (alpha string, beta
string) of occupied-orbital bit masks, ordered as
  |I> = prod_{p in alpha, ascending} a+_{p alpha} prod_{q in beta, ascending} a+_{q beta} |0>,
index I = i_alpha * n_beta_strings + i_beta.

Standard second-quantised notation is used internally:
  E_pq = sum_s a+_{ps} a_{qs},   gamma_pq = <E_pq>,
  Gamma_pqrs = sum_{st} <a+_{ps} a+_{rt} a_{st} a_{qs}>  (spins s, t)
             = <E_pq E_rs> - delta_qr gamma_ps,
  H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps).
The paper's RDMs (Sec. 2) are D^p_q = gamma_qp and P^{pq}_{sr} = Gamma_{sprq},
hence (D^-1)^o_p = (gamma^-1)_po and P^{qs}_{or} = Gamma_{oqrs}: the mean-field
term of Eq. orb_eom reads sum_o (gamma^-1)_po sum_qrs Gamma_oqrs W_rs phi_q.

Test infrastructure only (see the package docstring).
"""
import itertools

import numpy as np
import scipy.sparse as sp


def strings(n, k):
    """All bit masks of k occupied orbitals out of n, ascending by integer value."""
    out = []
    for occ in itertools.combinations(range(n), k):
        out.append(sum(1 << o for o in occ))
    return sorted(out)


def _excite(s, p, q):
    """a+_p a_q acting on string s: (new string, sign) or None."""
    if not (s >> q) & 1:
        return None
    sign = -1 if bin(s & ((1 << q) - 1)).count("1") % 2 else 1
    s1 = s & ~(1 << q)
    if (s1 >> p) & 1:
        return None
    if bin(s1 & ((1 << p) - 1)).count("1") % 2:
        sign = -sign
    return s1 | (1 << p), sign


class CISpace:
    def __init__(self, n, n_alpha, n_beta):
        self.n, self.na, self.nb = n, n_alpha, n_beta
        self.astr = strings(n, n_alpha)
        self.bstr = strings(n, n_beta)
        self.aidx = {s: i for i, s in enumerate(self.astr)}
        self.bidx = {s: i for i, s in enumerate(self.bstr)}
        self.dim = len(self.astr) * len(self.bstr)
        self.E = [[self._E(p, q) for q in range(n)] for p in range(n)]

    def index(self, sa, sb):
        return self.aidx[sa] * len(self.bstr) + self.bidx[sb]

    def _E(self, p, q):
        """Sparse matrix of E_pq = a+_{p alpha} a_{q alpha} + a+_{p beta} a_{q beta}.

        For the beta part the operators pass the n_alpha alpha creators twice,
        so only the sign inside the beta string remains.
        """
        rows, cols, vals = [], [], []
        nb = len(self.bstr)
        for ia, sa in enumerate(self.astr):
            for ib, sb in enumerate(self.bstr):
                J = ia * nb + ib
                r = _excite(sa, p, q)
                if r is not None:
                    rows.append(self.aidx[r[0]] * nb + ib)
                    cols.append(J)
                    vals.append(r[1])
                r = _excite(sb, p, q)
                if r is not None:
                    rows.append(ia * nb + self.bidx[r[0]])
                    cols.append(J)
                    vals.append(r[1])
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.dim, self.dim))

    def hamiltonian(self, h, eri):
        """Dense H_CI from one-electron h[p,q] and two-electron eri[p,q,r,s] = (pq|rs).

        Each term's sparse matrix is added into H at its nonzeros only (the
        same terms in the same order as adding the dense matrices, without
        forming a dense temporary per term)."""
        n = self.n
        H = np.zeros((self.dim, self.dim), dtype=np.complex128)

        def add(coef, M):
            M = M.tocoo()
            np.add.at(H, (M.row, M.col), coef * M.data)

        for p in range(n):
            for q in range(n):
                Epq = self.E[p][q]
                add(h[p, q], Epq)
                for r in range(n):
                    for s in range(n):
                        if eri[p, q, r, s] == 0:
                            continue
                        M = Epq @ self.E[r][s]
                        if q == r:
                            M = M - self.E[p][s]
                        add(0.5 * eri[p, q, r, s], M)
        return H

    def rdm1(self, C):
        n = self.n
        g = np.zeros((n, n), dtype=np.complex128)
        for p in range(n):
            for q in range(n):
                g[p, q] = np.vdot(C, self.E[p][q] @ C)
        return g

    def rdm2(self, C):
        """Gamma_pqrs = <E_pq E_rs> - delta_qr gamma_ps."""
        n = self.n
        g1 = self.rdm1(C)
        X = {(r, s): self.E[r][s] @ C for r in range(n) for s in range(n)}
        G = np.zeros((n, n, n, n), dtype=np.complex128)
        for p in range(n):
            for q in range(n):
                Y = self.E[q][p] @ C     # (E_pq)^dagger C
                for r in range(n):
                    for s in range(n):
                        G[p, q, r, s] = np.vdot(Y, X[(r, s)])
                        if q == r:
                            G[p, q, r, s] -= g1[p, s]
        return G
