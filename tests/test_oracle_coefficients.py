"""Pins of the KPM coefficient routines (App. B, Eqs. rho_KPM and F_KPM).

Each closed form is checked against an independent route: textbook Fourier
series, Chebyshev-Gauss quadrature (the paper's route for C_m), the Fejer
construction of the Jackson kernel, and the Chebyshev derivative identity that
links the step series to the grand-potential series.
"""
import numpy as np
import pytest

from oracle import kpm


def test_jackson_first_and_fejer_autocorrelation():
    for M in (1, 2, 7, 64, 257, 1024):
        g = kpm.jackson(M)
        assert g[0] == pytest.approx(1.0, abs=1e-14)
        # Jackson's kernel is the normalised autocorrelation of
        # a_nu = sin(pi (nu + 1)/(M + 1)), nu = 0..M-1 (Fejer-Riesz form).
        a = np.sin(np.pi * (np.arange(M) + 1) / (M + 1))
        ref = np.array([np.dot(a[: M - n], a[n:]) for n in range(M)]) / np.dot(a, a)
        assert np.max(np.abs(g - ref)) < 1e-13


def test_step_coefficients_square_wave_at_zero():
    # theta(-cos t) on [0, pi] = 1/2 - (2/pi) sum_k (-1)^k cos((2k+1) t)/(2k+1)
    M = 41
    c = kpm.step_coeffs(M, 0.0)
    ref = np.zeros(M)
    ref[0] = 0.5
    for k in range((M - 1) // 2 + 1):
        m = 2 * k + 1
        if m < M:
            ref[m] = (-1) ** (k + 1) / (m * np.pi)
    assert np.max(np.abs(c - ref)) < 1e-15


@pytest.mark.parametrize("x0", [-0.83, -0.2, 0.0, 0.37, 0.91])
def test_step_coefficients_vs_chebyshev_gauss(x0):
    M, K = 48, 1 << 18
    q = kpm.chebyshev_gauss(lambda x: (x < x0).astype(float), M, K)
    assert np.max(np.abs(kpm.step_coeffs(M, x0) - q)) < 4.0 / K


@pytest.mark.parametrize("x0", [-0.6, 0.0, 0.25, 0.8])
def test_omega_coefficients_vs_chebyshev_gauss(x0):
    M, K = 48, 1 << 16
    q = kpm.chebyshev_gauss(lambda x: np.minimum(x - x0, 0.0), M, K)
    assert np.max(np.abs(kpm.omega_coeffs(M, x0) - q)) < 20.0 / K ** 2


@pytest.mark.parametrize("x0", [-0.45, 0.0, 0.6])
def test_derivative_identity_links_both_series(x0):
    # d/dx min(x - x0, 0) = theta(x0 - x):  c'_{m-1} - c'_{m+1} = 2 m c^Omega_m
    M = 200
    cs = kpm.step_coeffs(M + 2, x0)
    co = kpm.omega_coeffs(M + 2, x0)
    m = np.arange(1, M)
    assert np.max(np.abs(cs[m - 1] - cs[m + 1] - 2 * m * co[m])) < 1e-15 * M


@pytest.mark.parametrize("M", [16, 128, 1024])
def test_jackson_damped_step_is_bounded(M):
    # The Jackson kernel is positive, so the damped step is a normalised
    # average of the step: values in [0, 1] (an undamped truncation overshoots
    # by the Gibbs 9%), and F(x) + F(-x) = 1 at x0 = 0.
    x = np.linspace(-1, 1, 4001)
    a = kpm.series(kpm.step_coeffs(M, 0.0), M)
    F = kpm.cheb_eval(a, x)
    assert F.min() > -1e-12 and F.max() < 1 + 1e-12
    assert np.max(np.abs(F + F[::-1] - 1.0)) < 1e-12
    raw = kpm.cheb_eval(kpm.series(kpm.step_coeffs(M, 0.0), M, damp=False), x)
    assert raw.max() > 1.05


def test_damped_series_converges_to_functions():
    x = np.array([-0.9, -0.5, -0.21, 0.19, 0.5, 0.93])
    x0 = 0.1
    prev = None
    for M in (64, 256, 1024, 4096):
        a = kpm.series(kpm.step_coeffs(M, x0), M)
        err = np.max(np.abs(kpm.cheb_eval(a, x) - (x < x0)))
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 1e-6
    ao = kpm.series(kpm.omega_coeffs(4096, x0), 4096)
    assert np.max(np.abs(kpm.cheb_eval(ao, x) - np.minimum(x - x0, 0))) < 1e-4


def test_cheb_eval_matches_cosine_definition():
    rng = np.random.default_rng(0)
    a = rng.normal(size=50)
    x = np.linspace(-1, 1, 101)
    ref = np.cos(np.arange(50)[:, None] * np.arccos(x)[None, :]).T @ a
    assert np.max(np.abs(kpm.cheb_eval(a, x) - ref)) < 1e-12
