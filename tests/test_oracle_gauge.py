"""Gauge pins of the oracle (Sec. II, App. A, B): covariance under a site
gauge transformation c_i -> e^{i theta_i} c_i, and magnetic translations on
a torus whose total flux makes a one-site translation gauge-equivalent.

Conventions fixed by readings N1-N4 (chi_ij = <c^dag_i c_j>, F_ij =
<c_i,up c_j,dn>) and by t_ij = t e^{i phi_ij} multiplying c^dag_i c_j:
theta sends phi_ij -> phi_ij + theta_i - theta_j, chi_ij -> e^{i(theta_j -
theta_i)} chi_ij, F_ij -> e^{i(theta_i + theta_j)} F_ij, n unchanged; W is
invariant and every observable transforms the same way.
"""
import math

import numpy as np
import pytest

from oracle import bdg, kpm, rmft
from oracle.lattice import peierls_phases
from paper_2212_05685_gb300 import inputs


def _gauge(model, theta, phi, p):
    N = model.N
    n, chi, F = rmft.split(p, N)
    phi2 = np.array(phi, dtype=np.float64, copy=True)
    chi2 = chi.copy()
    F2 = F.copy()
    for d in range(4):
        j = model.fwd[d]
        phi2[d] = phi[d] + theta - theta[j]
        chi2[:, d] = chi[:, d] * np.exp(1j * (theta[j] - theta))
    for e in range(4):
        j = model.nn4[e]
        F2[e] = F[e] * np.exp(1j * (theta + theta[j]))
    return phi2, rmft.join(n, chi2, F2)


def _observables(model, p, mu, M=96):
    fld = rmft.fields(model, p, mu)
    a, b = bdg.gershgorin(model, fld)
    F1, omega = kpm.f_spectral(bdg.dense(model, fld), a, b, M)
    return kpm.observables(model, F1), omega


@pytest.mark.parametrize("nx,ny,flux", [(6, 4, 1), (5, 5, 2)])
def test_site_gauge_covariance(nx, ny, flux):
    rng = np.random.default_rng(nx * 10 + ny)
    m0 = rmft.Model(nx, ny, flux=flux)
    p = inputs.random_params(nx, ny, 7)
    theta = rng.uniform(-math.pi, math.pi, size=nx * ny)
    phi2, p2 = _gauge(m0, theta, m0.phi, p)
    m2 = rmft.Model(nx, ny, flux=flux, phi=phi2)
    assert rmft.energy_W(m2, p2, 0.3) == pytest.approx(rmft.energy_W(m0, p, 0.3), abs=1e-12)
    o, om = _observables(m0, p, 0.3)
    o2, om2 = _observables(m2, p2, 0.3)
    _, expect = _gauge(m0, theta, m0.phi, o)
    assert np.max(np.abs(o2 - expect)) < 1e-12
    assert om2 == pytest.approx(om, abs=1e-10)
    # a wrong sign in any one rule breaks covariance (the pin is sensitive)
    _, wrong = _gauge(m0, -theta, m0.phi, o)
    assert np.max(np.abs(o2 - wrong)) > 1e-3


def _translate(p, nx, ny, sx, sy):
    """Order parameters of the cell moved by (sx, sy): value at i goes to i + s."""
    N = nx * ny
    n, chi, F = rmft.split(p, N)
    i = np.arange(N)
    src = ((i % nx - sx) % nx) + nx * ((i // nx - sy) % ny)
    return rmft.join(n[:, src], chi[:, :, src], F[:, src])


@pytest.mark.parametrize("sx,sy", [(1, 0), (0, 1), (1, 1)])
def test_magnetic_translation(sx, sy):
    """Total flux lcm(Nx, Ny) hc/e: a one-site translation changes the torus
    holonomies by multiples of 2 pi and so is a gauge transformation.  A cell
    whose only order parameters are (random, spin-equal) densities is then
    mapped onto itself by translation: n and |chi| move with the lattice."""
    nx, ny = 4, 6
    flux = 12
    model = rmft.Model(nx, ny, flux=flux)
    N = nx * ny
    rng = np.random.default_rng(3)
    n = 0.44 + 0.03 * rng.uniform(-1, 1, size=N)
    p = rmft.join(np.stack([n, n]), np.zeros((2, 4, N), complex), np.zeros((4, N), complex))
    o, om = _observables(model, p, 0.1)
    oT, omT = _observables(model, _translate(p, nx, ny, sx, sy), 0.1)
    moved = _translate(o, nx, ny, sx, sy)
    nT, chiT, FT = rmft.split(oT, N)
    nm, chim, Fm = rmft.split(moved, N)
    assert np.max(np.abs(nT - nm)) < 1e-12
    assert np.max(np.abs(np.abs(chiT) - np.abs(chim))) < 1e-12
    assert np.max(np.abs(FT)) < 1e-12
    assert omT == pytest.approx(om, abs=1e-10)


def test_translation_is_not_a_symmetry_at_one_flux_quantum():
    """Control: with one flux quantum a one-column translation changes the
    y holonomy by 2 pi / Nx, so the densities do not simply move."""
    nx, ny = 4, 6
    model = rmft.Model(nx, ny, flux=1)
    N = nx * ny
    rng = np.random.default_rng(3)
    n = 0.44 + 0.03 * rng.uniform(-1, 1, size=N)
    p = rmft.join(np.stack([n, n]), np.zeros((2, 4, N), complex), np.zeros((4, N), complex))
    o, _ = _observables(model, p, 0.1)
    oT, _ = _observables(model, _translate(p, nx, ny, 1, 0), 0.1)
    assert np.max(np.abs(oT[:N] - _translate(o, nx, ny, 1, 0)[:N])) > 1e-6
