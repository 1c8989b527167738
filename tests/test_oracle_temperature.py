"""Pins of the finite-temperature coefficients (App. B: C_m by Chebyshev-Gauss
quadrature of the Fermi and grand-potential functions)."""
import numpy as np
import pytest

from oracle import bdg, kpm, rmft
from paper_2212_05685_gb300 import inputs


def test_undamped_series_reproduce_the_functions():
    # analytic functions: the Chebyshev series converge exponentially
    a, b, T, M = 2.5, 0.1, 0.2, 512
    x = np.linspace(-0.999, 0.999, 801)
    c = kpm.chebyshev_gauss(lambda t: kpm.fermi(a * t + b, T), M, 4 * M)
    co = kpm.chebyshev_gauss(lambda t: kpm.grand(a * t + b, T) / a, M, 4 * M)
    assert np.max(np.abs(kpm.cheb_eval(kpm.series(c, M, damp=False), x) - kpm.fermi(a * x + b, T))) < 1e-10
    assert np.max(np.abs(kpm.cheb_eval(kpm.series(co, M, damp=False), x) - kpm.grand(a * x + b, T) / a)) < 1e-10


def test_grand_potential_is_the_antiderivative_of_the_occupation():
    eps = np.linspace(-3, 3, 61)
    T, h = 0.15, 1e-5
    d = (kpm.grand(eps + h, T) - kpm.grand(eps - h, T)) / (2 * h)
    assert np.max(np.abs(d - kpm.fermi(eps, T))) < 1e-9
    assert np.max(np.abs(kpm.grand(eps, 1e-4) - np.minimum(eps, 0.0))) < 1e-4


def test_particle_hole_symmetry_kills_even_terms():
    # f(e) + f(-e) = 1: at b = 0 the even coefficients vanish beyond m = 0
    am, _ = kpm.coefficients(256, 2.0, 0.0, T=0.05)
    assert am[0] == pytest.approx(0.5, abs=1e-14)
    assert np.max(np.abs(am[2::2])) < 1e-14


def test_low_temperature_approaches_the_step():
    M, a, b = 256, 2.3, -0.2
    a0, o0 = kpm.coefficients(M, a, b)
    errs = [np.max(np.abs(kpm.coefficients(M, a, b, T=T, K=64 * M)[0] - a0)) for T in (0.1, 0.03, 0.01, 0.003)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 0.02


def test_kpm_density_matrix_tends_to_exact_fermi():
    model = rmft.Model(6, 6)
    p = inputs.vortex_seed(inputs.Workload(6, 6, 0.125, inputs.two_vortex(6, 6), 64))
    fld = rmft.fields(model, p, 0.3)
    h = bdg.dense(model, fld)
    a, b = bdg.gershgorin(model, fld)
    T = 0.08
    F0, om0 = kpm.f_ed(h, T)
    errs, oerrs = [], []
    for M in (64, 128, 256, 512, 1024):
        F1, om1 = kpm.f_spectral(h, a, b, M, T)
        errs.append(np.max(np.abs(F1 - F0)))
        oerrs.append(abs(om1 - om0))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 2e-3 and oerrs[-1] < 1e-2 * abs(om0) * 1e-1
