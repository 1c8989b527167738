"""Local density of states (oracle; test infrastructure only).

App. C, Eqs. N_i and Gij: N_i(omega) = -Im G_ii(omega)/pi with
G_ii(omega) = sum_n [ g^t_{ii,up} |u_i^n|^2 / (omega - E_n + i Gamma)
                    + g^t_{ii,dn} |v_i^n|^2 / (omega + E_n + i Gamma) ],
u_i^n, v_i^n the (i, up) and (i, dn) Nambu components of eigenvector n of h,
Gamma = alpha |omega| + Gamma_0 the paper's Lorentzian broadening (alpha =
0.25, Gamma_0 = 3e-4).  Reading L1: g^t_{ii,sigma} = (g^t_{i sigma})^2 (the
bond factor g^t_i g^t_j at j = i); weights 1 give the plain BdG LDOS.  So the
spin-up part is the (i, up) spectral function at omega and the spin-down part
the (i, dn) spectral function at -omega.

Two routes:
  ldos_exact   the Lorentzians from the eigenpairs;
  ldos_cheb    the Chebyshev series of the resolvent truncated at M terms,
               1/(z - x) = (1/s) sum_m (2 - delta_m0) w^m T_m(x), z the
               rescaled complex energy, s = sqrt(z^2 - 1), w = z - s with
               |w| < 1, applied to the diagonal moments [T_m(h~)]_II (from
               the eigenpairs here); it tends to ldos_exact as |w|^M -> 0.
Output layout: [2][n_omega][N] (spin up, spin down).
"""
from __future__ import annotations

import numpy as np

from .rmft import site_factors, split


def gutzwiller_weights(params, N, gutzwiller=True):
    n, _, _ = split(params, N)
    return site_factors(n, gutzwiller)["gt"] ** 2


def _gamma(omega, alpha, gamma0):
    return alpha * np.abs(omega) + gamma0


def ldos_exact(h, omega, alpha=0.25, gamma0=3e-4, weights=None):
    E, U = np.linalg.eigh(h)
    D = h.shape[0]
    N = D // 2
    w2 = np.abs(U) ** 2
    out = np.empty((2, len(omega), N))
    for s in range(2):
        rows = w2[s::2]                      # (N, D): |U_{(i,s), n}|^2
        sign = 1.0 if s == 0 else -1.0
        for k, om in enumerate(omega):
            g = _gamma(om, alpha, gamma0)
            lor = (g / np.pi) / ((sign * om - E) ** 2 + g ** 2)
            out[s, k] = rows @ lor
    if weights is not None:
        out *= weights[:, None, :]
    return out


def resolvent_coeffs(z, M):
    """(2 - delta_m0) w^m / s for m < M, z complex rescaled (Im z > 0)."""
    s = np.sqrt(z * z - 1.0 + 0j)
    w = z - s
    if abs(w) > 1.0:
        s = -s
        w = z - s
    m = np.arange(M)
    c = 2.0 * w ** m / s
    c[0] *= 0.5
    return c


def ldos_from_moments(mu, a, b, omega, alpha=0.25, gamma0=3e-4, weights=None):
    """LDOS [2][n_omega][N] from diagonal moments mu[m][I] (M x D)."""
    M, D = mu.shape
    N = D // 2
    out = np.empty((2, len(omega), N))
    for s in range(2):
        sign = 1.0 if s == 0 else -1.0
        for k, om in enumerate(omega):
            g = _gamma(om, alpha, gamma0)
            z = (sign * om + 1j * g - b) / a
            G = resolvent_coeffs(z, M) @ mu[:, s::2] / a
            out[s, k] = -G.imag / np.pi
    if weights is not None:
        out *= weights[:, None, :]
    return out


def moments(h, a, b, M):
    """Diagonal moments [T_m(h~)]_II from the eigenpairs (M x D)."""
    E, U = np.linalg.eigh(h)
    x = (E - b) / a
    T = np.cos(np.arange(M)[:, None] * np.arccos(np.clip(x, -1.0, 1.0))[None, :])
    return T @ (np.abs(U) ** 2).T


def moments_probing(h, a, b, M, nx, ny, p, seed):
    """Probing estimate Re(conj(xi_J) [T_m(h~) r_colour(J)]_J) of the diagonal moments."""
    from .probing import probing_matrix
    E, U = np.linalg.eigh(h)
    x = (E - b) / a
    T = np.cos(np.arange(M)[:, None] * np.arccos(np.clip(x, -1.0, 1.0))[None, :])
    Z, xi = probing_matrix(nx, ny, p, seed)
    W = U.conj().T @ Z                        # (n, J)
    P = U.T * W                               # P[n, J] = U[J, n] W[n, J]
    return ((T @ P) * np.conj(xi)[None, :]).real


def ldos_cheb(h, a, b, M, omega, alpha=0.25, gamma0=3e-4, weights=None):
    mu = moments(h, a, b, M)
    return ldos_from_moments(mu, a, b, omega, alpha, gamma0, weights), mu
