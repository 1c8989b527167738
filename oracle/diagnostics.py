"""Vortex-profile order parameters (oracle; test infrastructure only).

Sec. III, Eq. giDelta: the physical pairing of site i,
    Delta_i = 1/8 sum_{sigma, tau} g^t_{i,i+tau,sigma} (-1)^{tau_y} Delta_{i,i+tau,sigma} x (bond phase),
tau = +-x, +-y, Delta_{ij,up} = F_ij and Delta_{ij,dn} = F_ji (reading N4),
g^t_{ij,sigma} = g^t_{i sigma} g^t_{j sigma}.  Reading D1: the bond phase is
taken as e^{+i phi_{i,i+tau}} in this code's convention (t_ij = t e^{i phi_ij}
multiplying c^dag_i c_j), the choice that makes Delta_i transform like a pair
at site i, e^{2 i theta_i}, under c_i -> e^{i theta_i} c_i; the printed sign of
the exponent depends on the hopping convention.

Eq. gm: the staggered magnetisation
    M_i = (-1)^{x+y} g^{s,xy}_i / 4 sum_tau sqrt(g^{s,z}_{i,i+tau} / g^{s,xy}_{i,i+tau}) m_i,
with g^{s,z}/g^{s,xy} = R of the bond (reading W3); where R < 0 (possible for
magnetic states away from a solution) the square root, and M_i, is NaN.
"""
from __future__ import annotations

import numpy as np

from .lattice import NN4, OPP
from .rmft import _bond_exchange, site_factors, split


def _bond_phase(model, e, j):
    """Peierls phase of the bond i -> i + e (e indexes NN4) for every site i."""
    if e == 0:
        return model.phi[0]
    if e == 1:
        return model.phi[1]
    return -model.phi[0 if e == 2 else 1][j]


def physical_pairing(model, params):
    N = model.N
    n, chi, F = split(params, N)
    gt = site_factors(n, model.gutzwiller)["gt"]
    out = np.zeros(N, dtype=np.complex128)
    for e, (dx, dy) in enumerate(NN4):
        j = model.nn4[e]
        sign = 1.0 if dy == 0 else -1.0
        ph = np.exp(1j * _bond_phase(model, e, j))
        out += sign * ph * (gt[0] * gt[0][j] * F[e] + gt[1] * gt[1][j] * F[OPP[e]][j])
    return out / 8.0


def staggered_magnetisation(model, params):
    N = model.N
    n, chi, F = split(params, N)
    sf = site_factors(n, model.gutzwiller)
    acc = np.zeros(N)
    for d in range(2):
        b = _bond_exchange(model, sf, n, chi, F, d)
        r = np.sqrt(b["R"])
        acc += r                      # bond (i, i + d)
        acc += r[model.nn4[d + 2]]    # bond (i - d, i), stored at i - d
    x, y = np.arange(N) % model.nx, np.arange(N) // model.nx
    return (-1.0) ** (x + y) * sf["gxy"] / 4.0 * acc * sf["m"]
