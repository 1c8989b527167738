"""Seeded synthetic inputs shaped like the paper's vortex-lattice workloads.

This module only draws seeded random numbers and lays them out; it holds none
of the method's arithmetic (no Gutzwiller factors, no Hamiltonian, no KPM).
Both the CUDA path and the CPU oracle consume the arrays it produces, so a
parity test always feeds identical inputs to both sides.

Workloads (Sec. II: square lattices with two hc/2e vortices per magnetic cell,
t'=-0.3t, J=0.3t, hole doping 0.125-0.24, Chebyshev orders M=1000-2000):

  cfg0  16x16, delta=0.125, vortices (4,8),(12,8),   M=256
  cfg1  48x24, delta=0.15,  vortices (12,12),(36,12), M=1024
  cfg2  100x100, delta=0.125, vortices (25,50),(75,50), M=2048, plus a
        bidirectional period-8 pair-density-wave term on the pairing seed
  cfg3  32 cells drawn from {24x12, 32x16, 48x24, 64x32}, delta~U[0.05,0.30]
  cfg4  64x64, delta=0.125, M=1024 (adjoint workload)

Order-parameter layout (float64, length 26*N, N = nx*ny, site i = x + nx*y):

  [0,   2N)   n[s][i]              s = 0 (up), 1 (down)
  [2N, 18N)   chi[s][d][i] complex  interleaved (re, im); d indexes the four
                                    forward bonds i -> i+d: +x, +y, +x+y, +x-y
  [18N,26N)   F[e][i] complex       F_{i,i+e} = <c_{i up} c_{i+e down}>,
                                    e = +x, +y, -x, -y

Seed recipe (one numpy PCG64 generator per seed, draws in this order):
  1. u_chi = uniform(-1, 1, size=(4, N))   one value per forward bond
  2. u_del = uniform(-1, 1, size=(2, N))   one value per nn bond (x, y)
  n_{i s} = (1 - delta)/2
  chi_{i,i+d,s} = 0.2 * (1 + 0.05 u_chi[d,i])            (both spins equal)
  Delta_b = sign_b * (0.1 * prod_v tanh(r_v/2) * exp(i sum_v theta_v)
                      * (1 + 0.1 u_del[b]) + pdw * (cos(2 pi X/8) + cos(2 pi Y/8)))
  with sign_b = +1 on x bonds, -1 on y bonds, (X, Y) the bond midpoint,
  (r_v, theta_v) its minimum-image polar coordinates about vortex v,
  and F_{i,j} = F_{j,i} = Delta_b on both orientations of the bond.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FWD = ((1, 0), (0, 1), (1, 1), (1, -1))   # forward bond directions d
NN4 = ((1, 0), (0, 1), (-1, 0), (0, -1))  # ordered nearest-neighbour pairs e
N_PARAM_PER_SITE = 26


@dataclasses.dataclass(frozen=True)
class Workload:
    nx: int
    ny: int
    delta: float
    vortices: tuple
    M: int
    seed: int = 0
    pdw: float = 0.0
    flux: int = 1          # total flux through the cell in units of hc/e
    t: float = 1.0
    tp: float = -0.3
    J: float = 0.3

    @property
    def n_sites(self) -> int:
        return self.nx * self.ny

    @property
    def dim(self) -> int:
        return 2 * self.nx * self.ny

    @property
    def n_target(self) -> float:
        return 1.0 - self.delta


def two_vortex(nx: int, ny: int):
    """Vortex centres at (nx/4, ny/2) and (3nx/4, ny/2)."""
    return ((nx // 4, ny // 2), ((3 * nx) // 4, ny // 2))


CFG0 = Workload(16, 16, 0.125, ((4, 8), (12, 8)), 256, seed=0)
CFG1 = Workload(48, 24, 0.15, ((12, 12), (36, 12)), 1024, seed=0)
CFG2 = Workload(100, 100, 0.125, two_vortex(100, 100), 2048, seed=0, pdw=0.02)
CFG4 = Workload(64, 64, 0.125, two_vortex(64, 64), 1024, seed=1)


def cfg3_cells(seed: int = 0, count: int = 32):
    """The uneven batch: shapes uniform over four cells, doping U[0.05, 0.30]."""
    rng = np.random.default_rng(seed)
    shapes = ((24, 12), (32, 16), (48, 24), (64, 32))
    pick = rng.integers(0, len(shapes), size=count)
    dop = rng.uniform(0.05, 0.30, size=count)
    out = []
    for k in range(count):
        nx, ny = shapes[int(pick[k])]
        out.append(Workload(nx, ny, float(dop[k]), two_vortex(nx, ny), 1024,
                            seed=seed + 1 + k))
    return out


def _min_image(d: float, L: int) -> float:
    return d - L * math.floor(d / L + 0.5)


def vortex_seed(w: Workload) -> np.ndarray:
    """Initial order parameters of a two-vortex cell (layout in the module doc)."""
    nx, ny, N = w.nx, w.ny, w.n_sites
    rng = np.random.default_rng(w.seed)
    u_chi = rng.uniform(-1.0, 1.0, size=(4, N))
    u_del = rng.uniform(-1.0, 1.0, size=(2, N))

    n = np.full((2, N), 0.5 * (1.0 - w.delta))
    chi = np.zeros((2, 4, N), dtype=np.complex128)
    chi[0] = 0.2 * (1.0 + 0.05 * u_chi)
    chi[1] = chi[0]
    F = np.zeros((4, N), dtype=np.complex128)
    for i in range(N):
        x, y = i % nx, i // nx
        for b, (dx, dy) in enumerate(((1, 0), (0, 1))):
            X, Y = x + 0.5 * dx, y + 0.5 * dy
            amp, theta = 1.0, 0.0
            for (vx, vy) in w.vortices:
                rx, ry = _min_image(X - vx, nx), _min_image(Y - vy, ny)
                amp *= math.tanh(math.hypot(rx, ry) / 2.0)
                theta += math.atan2(ry, rx)
            sign = 1.0 if b == 0 else -1.0
            val = 0.1 * amp * complex(math.cos(theta), math.sin(theta)) * (1.0 + 0.1 * u_del[b, i])
            if w.pdw:
                val += w.pdw * (math.cos(2 * math.pi * X / 8) + math.cos(2 * math.pi * Y / 8))
            val *= sign
            j = ((x + dx) % nx) + nx * ((y + dy) % ny)
            F[b, i] = val          # F_{i, i+b}
            F[b + 2, j] = val      # F_{j, j-b} = F_{i+b, i}
    return pack(n, chi, F)


def uniform_dwave(nx: int, ny: int, delta: float, chi_nn: float = 0.2,
                  chi_nnn: float = 0.05, pair: float = 0.1) -> np.ndarray:
    """Translation-invariant d-wave order parameters (F_x = -F_y)."""
    N = nx * ny
    n = np.full((2, N), 0.5 * (1.0 - delta))
    chi = np.zeros((2, 4, N), dtype=np.complex128)
    chi[:, 0:2, :] = chi_nn
    chi[:, 2:4, :] = chi_nnn
    F = np.zeros((4, N), dtype=np.complex128)
    F[0] = F[2] = pair
    F[1] = F[3] = -pair
    return pack(n, chi, F)


def random_params(nx: int, ny: int, seed: int, delta: float = 0.12,
                  spin_split: float = 0.0, scale: float = 1.0) -> np.ndarray:
    """Generic random order parameters (no symmetry), for convention tests."""
    rng = np.random.default_rng(seed)
    N = nx * ny
    base = 0.5 * (1.0 - delta)
    n = base + 0.03 * scale * rng.uniform(-1, 1, size=(2, N))
    if spin_split:
        n[0] += spin_split
        n[1] -= spin_split
    chi = 0.15 * scale * (rng.uniform(-1, 1, size=(2, 4, N)) + 1j * rng.uniform(-1, 1, size=(2, 4, N)))
    chi += 0.1
    F = 0.08 * scale * (rng.uniform(-1, 1, size=(4, N)) + 1j * rng.uniform(-1, 1, size=(4, N)))
    return pack(n, chi, F)


def target_density(w: Workload, seed: int, spread: float = 0.01) -> np.ndarray:
    """Per-site target densities 1 - delta + spread*U(-1,1) (adjoint loss)."""
    rng = np.random.default_rng(seed)
    return 1.0 - w.delta + spread * rng.uniform(-1.0, 1.0, size=w.n_sites)


def pack(n, chi, F) -> np.ndarray:
    N = n.shape[1]
    out = np.empty(N_PARAM_PER_SITE * N)
    out[0:2 * N] = np.asarray(n, dtype=np.float64).reshape(-1)
    out[2 * N:18 * N] = np.asarray(chi, dtype=np.complex128).reshape(-1).view(np.float64)
    out[18 * N:26 * N] = np.asarray(F, dtype=np.complex128).reshape(-1).view(np.float64)
    return out


def unpack(p: np.ndarray, N: int):
    p = np.ascontiguousarray(p, dtype=np.float64)
    n = p[0:2 * N].reshape(2, N)
    chi = p[2 * N:18 * N].view(np.complex128).reshape(2, 4, N)
    F = p[18 * N:26 * N].view(np.complex128).reshape(4, N)
    return n, chi, F
