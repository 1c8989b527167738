"""Pins of the vortex-profile order parameters (Eqs. giDelta, gm; reading D1)."""
import math

import numpy as np
import pytest

from oracle import diagnostics, rmft
from paper_2212_05685_gb300 import inputs


def test_uniform_dwave_closed_form():
    # F_x = -F_y = D0, uniform density, no field: Delta_i = (g^t)^2 D0 = 2 delta/(1+delta) D0
    delta, D0 = 0.125, 0.1
    model = rmft.Model(6, 6, flux=0)
    p = inputs.uniform_dwave(6, 6, delta, pair=D0)
    d = diagnostics.physical_pairing(model, p)
    assert np.max(np.abs(d - 2 * delta / (1 + delta) * D0)) < 1e-14


def test_gauge_covariance_of_the_pairing():
    nx, ny = 6, 4
    m0 = rmft.Model(nx, ny, flux=1)
    p = inputs.random_params(nx, ny, 3)
    theta = np.random.default_rng(2).uniform(-math.pi, math.pi, nx * ny)
    n, chi, F = rmft.split(p, nx * ny)
    phi2 = m0.phi.copy()
    F2 = F.copy()
    for d in range(4):
        phi2[d] = m0.phi[d] + theta - theta[m0.fwd[d]]
    for e in range(4):
        F2[e] = F[e] * np.exp(1j * (theta + theta[m0.nn4[e]]))
    m2 = rmft.Model(nx, ny, flux=1, phi=phi2)
    d0 = diagnostics.physical_pairing(m0, p)
    d2 = diagnostics.physical_pairing(m2, rmft.join(n, chi, F2))
    assert np.max(np.abs(d2 - np.exp(2j * theta) * d0)) < 1e-14


def test_staggered_magnetisation():
    nx, ny = 4, 4
    model = rmft.Model(nx, ny, flux=0)
    N = nx * ny
    # m = 0: no magnetisation
    assert np.max(np.abs(diagnostics.staggered_magnetisation(model, inputs.uniform_dwave(nx, ny, 0.1)))) == 0.0
    # Neel order without bonds (chi = F = 0): R = X^2, so M_i = (-1)^{x+y} g^xy_i |X| m_i
    x, y = np.arange(N) % nx, np.arange(N) // nx
    st = (-1.0) ** (x + y)
    ms = 0.05
    n = np.stack([0.45 + st * ms, 0.45 - st * ms])
    p = rmft.join(n, np.zeros((2, 4, N), complex), np.zeros((4, N), complex))
    M = diagnostics.staggered_magnetisation(model, p)
    delta, m = 1 - 0.9, st * ms
    P = 1 - delta ** 2 + 4 * ms ** 2
    gxy = 2 * (1 - delta) / P
    X = 1 + 12 * (1 - delta) ** 2 / P
    assert np.max(np.abs(M - st * gxy * X * m)) < 1e-13
