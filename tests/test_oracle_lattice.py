"""Pins of the Peierls phases (Sec. II, App. C: A = B(0, x), B = 2 Phi0/(Nx Ny)).

Gauge-invariant content of a lattice gauge field: every plaquette flux, the
half-plaquette flux of each next-nearest-neighbour triangle, and the
holonomies around the two cycles of the torus.
"""
import numpy as np
import pytest

from oracle.lattice import FWD, peierls_phases, site


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


@pytest.mark.parametrize("nx,ny,flux", [(16, 16, 1), (48, 24, 1), (5, 7, 1), (6, 4, 3), (3, 3, 1)])
def test_every_plaquette_encloses_the_same_flux(nx, ny, flux):
    phi = peierls_phases(nx, ny, flux)
    f = 2 * np.pi * flux / (nx * ny)
    for x in range(nx):
        for y in range(ny):
            i = site(x, y, nx, ny)
            ix = site(x + 1, y, nx, ny)
            iy = site(x, y + 1, nx, ny)
            # counter-clockwise: +x at y, +y at x+1, back along +x at y+1, down +y at x
            circ = phi[0, i] + phi[1, ix] - phi[0, iy] - phi[1, i]
            assert _wrap(circ + f) == pytest.approx(0.0, abs=1e-12)
            # lower-right triangle (x,y)->(x+1,y)->(x+1,y+1)->(x,y): half the flux
            tri = phi[0, i] + phi[1, ix] - phi[2, i]
            assert _wrap(tri + 0.5 * f) == pytest.approx(0.0, abs=1e-12)
            # triangle (x,y)->(x+1,y-1)->(x+1,y)->(x,y) (counter-clockwise)
            idn = site(x + 1, y - 1, nx, ny)
            tri2 = phi[3, i] + phi[1, idn] - phi[0, i]
            assert _wrap(tri2 + 0.5 * f) == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("nx,ny,flux", [(16, 16, 1), (12, 8, 2)])
def test_total_flux_and_holonomies(nx, ny, flux):
    phi = peierls_phases(nx, ny, flux)
    f = 2 * np.pi * flux / (nx * ny)
    # Wilson loop along x at row y: phase 2 pi flux y / Ny (magnetic boundary condition)
    for y in range(ny):
        wx = sum(phi[0, site(x, y, nx, ny)] for x in range(nx))
        assert _wrap(wx - 2 * np.pi * flux * y / ny) == pytest.approx(0.0, abs=1e-12)
    # Wilson loop along y at column x: -Ny * f * x
    for x in range(nx):
        wy = sum(phi[1, site(x, y, nx, ny)] for y in range(ny))
        assert _wrap(wy + ny * f * x) == pytest.approx(0.0, abs=1e-12)
    # flux of hc/e per quantum: B = 2 Phi0/(Nx Ny) per plaquette times Nx Ny
    assert f * nx * ny == pytest.approx(2 * np.pi * flux)


def test_zero_flux_has_no_phases():
    assert np.all(peierls_phases(8, 6, 0) == 0.0)


def test_y_bond_phase_is_landau_gauge():
    nx, ny = 10, 6
    phi = peierls_phases(nx, ny, 1)
    for x in range(nx):
        for y in range(ny):
            assert phi[1, site(x, y, nx, ny)] == pytest.approx(-2 * np.pi * x / (nx * ny))
            if x < nx - 1:
                assert phi[0, site(x, y, nx, ny)] == 0.0
                assert phi[2, site(x, y, nx, ny)] == pytest.approx(-2 * np.pi * (x + 0.5) / (nx * ny))
