"""Naive-KPM columns of one Hamiltonian on spawn-started worker processes.

TEST INFRASTRUCTURE ONLY (tests, and the benchmark's CPU-baseline leg).  Every
worker builds the oracle's fields, Gershgorin bounds and CSR Nambu matrix of
the same order parameters once, then runs the naive Chebyshev recursion of
Eq. alpha (`kpm.f_naive`) on the unit columns it is given: columns are
independent recursions (App. B), so a sample of them splits over processes
without changing any column's arithmetic.  Workers are started with `spawn`,
so a pool may be created after CUDA was initialised in the parent.
"""
from __future__ import annotations

import multiprocessing as mp
import time

import numpy as np

_W = {}


def _init(nx, ny, flux, params, mu, M):
    from . import bdg, rmft
    model = rmft.Model(nx, ny, flux=flux)
    f = rmft.fields(model, np.asarray(params), mu)
    a, b = bdg.gershgorin(model, f)
    _W.update(model=model, h=bdg.csr(model, f), a=a, b=b, M=M)


def _run_cols(cols):
    from . import kpm
    t0 = time.perf_counter()
    kpm.f_naive(_W["h"], _W["a"], _W["b"], _W["M"], cols=np.asarray(cols))
    return time.perf_counter() - t0


def _run_sites(sites):
    from . import kpm
    t0 = time.perf_counter()
    sites = np.asarray(sites)
    cols = np.sort(np.concatenate([2 * sites, 2 * sites + 1]))
    Fc, _ = kpm.f_naive(_W["h"], _W["a"], _W["b"], _W["M"], cols=cols)
    n, chi, F = kpm.observables_at(_W["model"], Fc, cols, sites)
    return time.perf_counter() - t0, n, chi, F


class ColumnPool:
    """Worker processes holding the Nambu matrix of (nx, ny, params, mu)."""

    def __init__(self, nx, ny, params, mu, M, workers, flux=1):
        self.workers = int(workers)
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_init,
                                                 initargs=(nx, ny, flux, np.asarray(params), float(mu), M))
        self.pool.map(_run_cols, [[0]] * self.workers)  # every worker initialised

    def time_columns(self, col_lists):
        """Wall time of the workers on the given column lists (one list per task)."""
        t0 = time.perf_counter()
        self.pool.map(_run_cols, col_lists)
        return time.perf_counter() - t0

    def site_observables(self, sites):
        """(n (2, k), chi (2, 4, k), F (4, k), wall seconds) of the sites,
        split evenly over the workers."""
        sites = np.asarray(sites)
        chunks = [c for c in np.array_split(sites, self.workers) if len(c)]
        t0 = time.perf_counter()
        res = self.pool.map(_run_sites, [c.tolist() for c in chunks])
        dt = time.perf_counter() - t0
        n = np.concatenate([r[1] for r in res], axis=1)
        chi = np.concatenate([r[2] for r in res], axis=2)
        F = np.concatenate([r[3] for r in res], axis=1)
        return n, chi, F, dt

    def close(self):
        self.pool.close()
        self.pool.join()


def sample_sites(nx, ny, count, centres, seed=0):
    """`count` distinct sites: the given centres and their four neighbours
    first, then uniformly drawn others."""
    picked = []
    for (x, y) in centres:
        for dx, dy in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
            i = (x + dx) % nx + nx * ((y + dy) % ny)
            if i not in picked:
                picked.append(i)
    rng = np.random.default_rng(seed)
    rest = [int(i) for i in rng.permutation(nx * ny) if int(i) not in picked]
    return np.array(sorted(picked + rest[:max(0, count - len(picked))]))
