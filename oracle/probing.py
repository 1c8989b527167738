"""Probing estimate of the KPM density matrix (oracle; test infrastructure only).

App. B: the moments are estimated with R correlated random vectors (the
probing method of the paper's refs. Silver94, Tang12) instead of all D unit
vectors.  Reading P2 (the paper gives no colouring): the Nambu rows
K = 2 i + alpha of site i = (x, y) are coloured

    colour(K) = alpha + 2 ((x mod p) + p (y mod p)),   R = 2 p^2 colours,

(p divides Nx and Ny), so rows of one colour are p sites apart in x and y and
a row's colour differs from that of every row within one site of it except
itself.  Probing vector r_c has entries xi_K on the rows of colour c and 0
elsewhere, with phases xi_K = exp(2 pi i u_K) from the counter-based
generator SplitMix64 (Steele, Lea and Flood 2014):

    z = x + 0x9E3779B97F4A7C15;  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB;  z ^ (z >> 31)   (mod 2^64),

x = seed * 2^32 + K, u_K = (z >> 11) * 2^-53.  The estimate of column J of
F_M(h~) is conj(xi_J) F_M(h~) r_colour(J): exact on row J itself and on the
rows whose colour differs from all other rows of colour(J) within reach,
contaminated by F_M(h~)_{K J'} for the other rows J' of the same colour.  The
grand potential uses the same estimate of the diagonal of G_M(h~).
"""
from __future__ import annotations

import numpy as np

from .kpm import cheb_eval, coefficients, observables

_MASK = (1 << 64) - 1


def splitmix64(x):
    z = (x + 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def phases(D, seed):
    """xi_K, K = 0..D-1."""
    u = np.array([(splitmix64((seed << 32) + K) >> 11) * 2.0 ** -53 for K in range(D)])
    return np.exp(2j * np.pi * u)


def colours(nx, ny, p):
    assert nx % p == 0 and ny % p == 0 and p >= 2
    K = np.arange(2 * nx * ny)
    i, alpha = K // 2, K % 2
    x, y = i % nx, i // nx
    return alpha + 2 * ((x % p) + p * (y % p))


def probing_matrix(nx, ny, p, seed):
    """Z with Z[:, J] = r_colour(J) (D x D)."""
    c = colours(nx, ny, p)
    xi = phases(2 * nx * ny, seed)
    Z = (c[:, None] == c[None, :]) * xi[:, None]
    return Z, xi


def f_probing(h, a, b, M, nx, ny, p, seed, T=0.0):
    """(estimate of F_M(h~) column by column, estimate of Omega_M)."""
    E, U = np.linalg.eigh(h)
    x = (E - b) / a
    am, ao = coefficients(M, a, b, T)
    Z, xi = probing_matrix(nx, ny, p, seed)
    FZ = (U * cheb_eval(am, x)) @ (U.conj().T @ Z)
    Fest = FZ * np.conj(xi)[None, :]
    GZ = (U * cheb_eval(ao, x)) @ (U.conj().T @ Z)
    omega = float(a * np.sum((np.diag(GZ) * np.conj(xi)).real))
    return Fest, omega


def observables_probing(model, h, a, b, M, p, seed, T=0.0):
    F, omega = f_probing(h, a, b, M, model.nx, model.ny, p, seed, T)
    return observables(model, F), omega


def columns_probing_naive(hcsr, a, b, M, nx, ny, p, seed, cols_of):
    """Probing estimates of the columns of F_M(h~) whose row has one of the
    given colours, by the Chebyshev recursion on those probing vectors (for
    large lattices): returns (J, F) with F[:, k] = conj(xi_J) F_M(h~) r_colour(J)
    for the rows J of those colours."""
    import scipy.sparse as sps
    D = hcsr.shape[0]
    cl = colours(nx, ny, p)
    xi = phases(D, seed)
    cols_of = np.asarray(cols_of)
    R = np.zeros((D, len(cols_of)), dtype=np.complex128)
    for k, col in enumerate(cols_of):
        rows = np.nonzero(cl == col)[0]
        R[rows, k] = xi[rows]
    ht = (hcsr - b * sps.identity(D, dtype=np.complex128, format="csr")) / a
    am, _ = coefficients(M, a, b)
    V0 = R
    acc = am[0] * V0
    if M > 1:
        V1 = ht @ V0
        acc = acc + am[1] * V1
        for m in range(2, M):
            V0, V1 = V1, 2.0 * (ht @ V1) - V0
            acc = acc + am[m] * V1
    J = np.nonzero(np.isin(cl, cols_of))[0]
    idx = {int(col): k for k, col in enumerate(cols_of)}
    F = np.stack([np.conj(xi[j]) * acc[:, idx[int(cl[j])]] for j in J], axis=1)
    return J, F
