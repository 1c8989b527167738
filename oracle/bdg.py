"""Nambu (BdG) matrix of the effective Hamiltonian (oracle; test infrastructure only).

App. B: with the Nambu spinor d_i = (c_{i up}, c^dagger_{i dn}) the effective
Hamiltonian is H_eff = sum_IJ h_IJ d^dagger_I d_J with I = (i, alpha), here
flattened as I = 2 i + alpha.  The entries are the derivatives h_IJ = dW/drho_IJ
of W with respect to rho_IJ = <d^dagger_I d_J> (Eq. for rho = dE/dh), which in
terms of the fields eps = dW/dn, T = dW/dchi and D = dW/dF* reads

  h[(i,0),(i,0)] = eps_{i up}          h[(i,1),(i,1)] = -eps_{i dn}
  h[(i,0),(j,0)] = T_{ij up}           h[(i,1),(j,1)] = -conj(T_{ij dn})
  h[(i,0),(j,1)] = -D_{ij}             (ordered nn pairs i -> j = i+e)

and Hermitian conjugates.  (Readings N1-N4: the printed lower-left block
D*_{ji dn}, the sign of the site term and the sign of the pairing entry are
fixed here by rho_IJ = <d^dagger_I d_J> and h_IJ = dW/drho_IJ.)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .rmft import split


def entries(model, fld):
    """COO triplets (rows, cols, vals) of h, Hermitian conjugates included."""
    N = model.N
    eps, T, D = split(fld, N)
    i = np.arange(N)
    rows, cols, vals = [2 * i, 2 * i + 1], [2 * i, 2 * i + 1], [eps[0].astype(np.complex128), -eps[1].astype(np.complex128)]
    for d in range(4):
        j = model.fwd[d]
        rows += [2 * i, 2 * j, 2 * i + 1, 2 * j + 1]
        cols += [2 * j, 2 * i, 2 * j + 1, 2 * i + 1]
        vals += [T[0, d], np.conj(T[0, d]), -np.conj(T[1, d]), -T[1, d]]
    for e in range(4):
        j = model.nn4[e]
        rows += [2 * i, 2 * j + 1]
        cols += [2 * j + 1, 2 * i]
        vals += [-D[e], -np.conj(D[e])]
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def dense(model, fld):
    r, c, v = entries(model, fld)
    h = np.zeros((2 * model.N, 2 * model.N), dtype=np.complex128)
    np.add.at(h, (r, c), v)
    return h


def csr(model, fld):
    r, c, v = entries(model, fld)
    D = 2 * model.N
    return sp.coo_matrix((v, (r, c)), shape=(D, D)).tocsr()


def gershgorin(model, fld, margin=0.01):
    """Spectral bounds from Gershgorin discs of the 13-entry rows.

    R_I is the sum of the moduli of the 12 off-diagonal stencil entries of row
    I (entries that land on the same column on tiny tori are not merged; the
    bound stays valid).  Returns (a, b): h~ = (h - b)/a, with the half-width
    widened by `margin` (1%).
    """
    N = model.N
    eps, T, D = split(fld, N)
    R = np.zeros((2, N))
    for d in range(4):
        j = model.fwd[d]
        for s in range(2):
            R[s] += np.abs(T[s, d])
            np.add.at(R[s], j, np.abs(T[s, d]))
    for e in range(4):
        j = model.nn4[e]
        R[0] += np.abs(D[e])
        np.add.at(R[1], j, np.abs(D[e]))
    diag = np.stack([eps[0], -eps[1]])
    emax = float(np.max(diag + R))
    emin = float(np.min(diag - R))
    b = 0.5 * (emax + emin)
    half = 0.5 * (emax - emin)
    # a single-point spectrum (no off-diagonal entries, flat diagonal) has
    # half-width 0: any a > 0 rescales it, take 1
    a = (1.0 + margin) * half if half > 0.0 else 1.0
    return a, b
