"""Square-lattice geometry and Peierls phases (oracle; test infrastructure only).

Sec. II: t_ij -> t e^{i phi_ij}, phi_ij = -(pi/Phi0) * integral_{r_i}^{r_j} A.dr,
Landau gauge A = B (0, x).  App. C: B = 2 Phi0 / (Nx Ny), i.e. flux hc/e through
the cell.  With `flux` quanta of hc/e the phase per unit of integral x dy is
f = 2 pi flux / (Nx Ny).

Readings (the paper is silent on these):
  * next-nearest-neighbour bonds use the straight-line integral;
  * Landau gauge is not periodic in x: a bond that crosses the x boundary
    carries the magnetic-translation phase 2 pi flux y'/Ny (y' the row it
    lands on), so that every plaquette of the torus, wrap plaquettes included,
    encloses the same flux.
"""
from __future__ import annotations

import numpy as np

FWD = ((1, 0), (0, 1), (1, 1), (1, -1))   # forward bonds d: +x, +y, +x+y, +x-y
NN4 = ((1, 0), (0, 1), (-1, 0), (0, -1))  # ordered nn pairs e: +x, +y, -x, -y
OPP = (2, 3, 0, 1)                        # e -> -e


def site(x, y, nx, ny):
    return (x % nx) + nx * (y % ny)


def coords(nx, ny):
    i = np.arange(nx * ny)
    return i % nx, i // nx


def bond_phase(x, y, dx, dy, nx, ny, flux=1):
    """phi for the bond (x, y) -> (x+dx, y+dy), dx in {0, 1}."""
    f = 2.0 * np.pi * flux / (nx * ny)
    # -(pi/Phi0) * B * integral x dy along the straight segment
    phi = -f * dy * (x + 0.5 * dx)
    if x + dx >= nx:  # landed across the x boundary: magnetic translation
        phi = phi + 2.0 * np.pi * flux * ((y + dy) % ny) / ny
    return phi


def peierls_phases(nx, ny, flux=1):
    """phi[d][i] for the four forward bonds of every site (float64, 4 x N)."""
    x, y = coords(nx, ny)
    out = np.empty((4, nx * ny))
    for d, (dx, dy) in enumerate(FWD):
        out[d] = [bond_phase(int(a), int(b), dx, dy, nx, ny, flux) for a, b in zip(x, y)]
    return out


def neighbour(i, dx, dy, nx, ny):
    return site(i % nx + dx, i // nx + dy, nx, ny)


def neighbour_table(nx, ny, dirs):
    x, y = coords(nx, ny)
    return np.stack([site(x + dx, y + dy, nx, ny) for (dx, dy) in dirs])
