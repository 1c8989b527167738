"""Many-body brute force on a few sites (oracle; test infrastructure only).

Builds the fermion operators of 2L spin orbitals by the Jordan-Wigner
construction, writes H_eff = sum_IJ h_IJ d^dagger_I d_J with the Nambu
operators of App. B (d_{i,0} = c_{i up}, d_{i,1} = c^dagger_{i dn}) as a sparse
Fock-space matrix, finds its ground state by Lanczos, and evaluates
correlation functions straight from the many-body state.  Nothing here uses
the single-particle matrix function f(h), so it pins the readings N1-N4 and
the Wick decomposition W2 independently.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def fermion_ops(n_modes):
    """Annihilation operators c_k (k = 0..n_modes-1) as CSR matrices."""
    a = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    Z = sp.csr_matrix(np.diag([1.0, -1.0]))
    I = sp.identity(2, format="csr")
    ops = []
    for k in range(n_modes):
        m = sp.identity(1, format="csr")
        for l in range(n_modes):
            m = sp.kron(m, Z if l < k else (a if l == k else I), format="csr")
        ops.append(m.astype(np.complex128))
    return ops


class Cluster:
    """L sites, modes ordered k = 2 i + s (s = 0 up, 1 down)."""

    def __init__(self, L):
        self.L = L
        self.c = fermion_ops(2 * L)
        self.cd = [op.getH().tocsr() for op in self.c]

    def d(self, I):
        i, al = divmod(I, 2)
        return self.c[2 * i] if al == 0 else self.cd[2 * i + 1]

    def ddag(self, I):
        i, al = divmod(I, 2)
        return self.cd[2 * i] if al == 0 else self.c[2 * i + 1]

    def hamiltonian(self, h):
        D = 2 * self.L
        H = None
        for I in range(D):
            for J in range(D):
                if h[I, J] != 0:
                    t = h[I, J] * (self.ddag(I) @ self.d(J))
                    H = t if H is None else H + t
        return H.tocsr()

    def ground_state(self, h):
        H = self.hamiltonian(h)
        if H.shape[0] <= 512:
            w, v = np.linalg.eigh(H.toarray())
            return v[:, 0], w[:2]
        # shift-invert about a point below the spectrum (sum of |h_IJ| bounds
        # |E| for every many-body state); plain 'SA' Lanczos can miss an
        # isolated ground state of one fermion-parity sector
        sigma = -float(np.sum(np.abs(h))) - 1.0
        w, v = spla.eigsh(H, k=2, sigma=sigma, which="LM", tol=1e-13)
        order = np.argsort(w)
        return v[:, order[0]], w[order]

    @staticmethod
    def ev(psi, op):
        return np.vdot(psi, op @ psi)

    def rho_nambu(self, psi):
        """<d^dagger_I d_J> evaluated in the many-body state."""
        D = 2 * self.L
        out = np.empty((D, D), dtype=np.complex128)
        for I in range(D):
            for J in range(D):
                out[I, J] = self.ev(psi, self.ddag(I) @ self.d(J))
        return out

    def hop(self, psi, i, j, s):
        """<c^dagger_{i s} c_{j s}>"""
        return self.ev(psi, self.cd[2 * i + s] @ self.c[2 * j + s])

    def pair(self, psi, i, j):
        """<c_{i up} c_{j dn}>"""
        return self.ev(psi, self.c[2 * i] @ self.c[2 * j + 1])

    def spin_corr(self, psi, i, j):
        """(<S^z_i S^z_j>, <(S^+_i S^-_j + S^-_i S^+_j)/2>) with S = (1/2) c^dag sigma c."""
        nu_i = self.cd[2 * i] @ self.c[2 * i]
        nd_i = self.cd[2 * i + 1] @ self.c[2 * i + 1]
        nu_j = self.cd[2 * j] @ self.c[2 * j]
        nd_j = self.cd[2 * j + 1] @ self.c[2 * j + 1]
        szz = self.ev(psi, 0.25 * (nu_i - nd_i) @ (nu_j - nd_j)).real
        sp_i = self.cd[2 * i] @ self.c[2 * i + 1]
        sm_j = self.cd[2 * j + 1] @ self.c[2 * j]
        sm_i = self.cd[2 * i + 1] @ self.c[2 * i]
        sp_j = self.cd[2 * j] @ self.c[2 * j + 1]
        sxy = self.ev(psi, 0.5 * (sp_i @ sm_j + sm_i @ sp_j)).real
        return szz, sxy
