"""Zero-field translation-invariant case in momentum space (oracle).

TEST INFRASTRUCTURE ONLY.  With flux 0 and identical fields on every site the
Nambu matrix of App. B is block diagonal in crystal momentum k: plane waves
psi_{(i, alpha)} = e^{i k.r_i} u_alpha / sqrt(N) give the 2 x 2 blocks

  h_k[0,0] =  eps_up + sum_d (T_{d up} e^{i k.d} + c.c.)
  h_k[1,1] = -eps_dn - sum_d (T_{d dn} e^{-i k.d} + c.c.)
  h_k[0,1] = -sum_e D_e e^{i k.e},   h_k[1,0] = conj(h_k[0,1])

(d over the four forward bonds, e over the four ordered nn pairs).  A matrix
polynomial acts block by block, so F_M(h~) restricted to momentum k is
F_M(h~_k), and the real-space entries follow by one Fourier sum:

  f(h)_{(j+r, alpha), (j, beta)} = (1/N) sum_k e^{i k.r} [F_M(h~_k)]_{alpha beta}.

This costs O(N M), so it reaches the full 100 x 100 lattice and pins the
Chebyshev recursion at the size the benchmark runs.
"""
from __future__ import annotations

import numpy as np

from .kpm import cheb_eval, coefficients
from .lattice import FWD, NN4
from .rmft import join, split


def blocks(nx, ny, fld_site):
    """h_k for every k of the nx x ny grid; fld_site = (eps[2], T[2][4], D[4])."""
    eps, T, D = fld_site
    kx = 2.0 * np.pi * np.arange(nx) / nx
    ky = 2.0 * np.pi * np.arange(ny) / ny
    KX, KY = np.meshgrid(kx, ky, indexing="xy")
    KX, KY = KX.reshape(-1), KY.reshape(-1)
    hk = np.zeros((KX.size, 2, 2), dtype=np.complex128)
    hk[:, 0, 0] = eps[0]
    hk[:, 1, 1] = -eps[1]
    for d, (dx, dy) in enumerate(FWD):
        ph = np.exp(1j * (KX * dx + KY * dy))
        hk[:, 0, 0] += 2.0 * (T[0][d] * ph).real
        hk[:, 1, 1] -= 2.0 * (T[1][d] * np.conj(ph)).real
    for e, (dx, dy) in enumerate(NN4):
        ph = np.exp(1j * (KX * dx + KY * dy))
        hk[:, 0, 1] += -D[e] * ph
    hk[:, 1, 0] = np.conj(hk[:, 0, 1])
    return KX, KY, hk


def kpm_uniform(nx, ny, fld_site, a, b, M):
    """Order parameters and Omega_M of a uniform zero-field state, KPM at order M.

    fld_site: the fields of one site (all sites equal).  Returns (params, Omega)
    in the flat layout of rmft.py (every site identical).
    """
    N = nx * ny
    KX, KY, hk = blocks(nx, ny, fld_site)
    lam, U = np.linalg.eigh(hk)
    x = (lam - b) / a
    am, ao = coefficients(M, a, b)
    Fx = cheb_eval(am, x.reshape(-1)).reshape(x.shape)
    Gx = cheb_eval(ao, x.reshape(-1)).reshape(x.shape)
    Fk = np.einsum("kan,kn,kbn->kab", U, Fx, np.conj(U))

    def entry(dx, dy, al, be):
        return np.sum(np.exp(1j * (KX * dx + KY * dy)) * Fk[:, al, be]) / N

    n = np.empty((2, N))
    chi = np.empty((2, 4, N), dtype=np.complex128)
    F = np.empty((4, N), dtype=np.complex128)
    n[0] = entry(0, 0, 0, 0).real
    n[1] = 1.0 - entry(0, 0, 1, 1).real
    for d, (dx, dy) in enumerate(FWD):
        chi[0, d] = entry(dx, dy, 0, 0)
        chi[1, d] = -np.conj(entry(dx, dy, 1, 1))
    for e, (dx, dy) in enumerate(NN4):
        F[e] = -np.conj(entry(dx, dy, 1, 0))
    return join(n, chi, F), float(a * np.sum(Gx))


def site_fields(fld, N, i=0):
    eps, T, D = split(fld, N)
    return eps[:, i].copy(), T[:, :, i].copy(), D[:, i].copy()
