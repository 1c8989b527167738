"""Pins of the probing estimate (App. B; reading P2): singleton colours give
the exact trace, the estimate is unbiased over the random phases, and its
error falls as same-colour rows move apart; the phase generator matches the
published SplitMix64 reference outputs."""
import numpy as np
import pytest

from oracle import bdg, kpm, probing, rmft
from paper_2212_05685_gb300 import inputs


def test_splitmix64_reference_values():
    # first outputs of the SplitMix64 stream seeded with 1234567 (state advanced
    # by the golden-ratio increment before each output), as published with the
    # generator's reference implementation
    state = 1234567
    out = []
    for _ in range(5):
        out.append(probing.splitmix64(state))
        state = (state + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
                   16408922859458223821]


def _cell(nx, ny, seed=0):
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64, seed=seed)
    model = rmft.Model(nx, ny)
    fld = rmft.fields(model, inputs.vortex_seed(w), 0.3)
    h = bdg.dense(model, fld)
    a, b = bdg.gershgorin(model, fld)
    return model, h, a, b


def test_colouring_separates_local_rows():
    nx, ny, p = 6, 6, 3
    c = probing.colours(nx, ny, p)
    model = rmft.Model(nx, ny)
    for i in range(nx * ny):
        x, y = i % nx, i // nx
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                j = ((x + dx) % nx) + nx * ((y + dy) % ny)
                for al in (0, 1):
                    for be in (0, 1):
                        same = c[2 * i + al] == c[2 * j + be]
                        assert same == (i == j and al == be)


def test_singleton_colours_are_the_exact_trace():
    nx = ny = 4
    model, h, a, b = _cell(nx, ny)
    M = 80
    exact, om = kpm.f_spectral(h, a, b, M)
    est, om_est = probing.f_probing(h, a, b, M, nx, ny, 4, seed=3)  # p = nx: one site per colour
    assert np.max(np.abs(est - exact)) < 1e-12
    assert om_est == pytest.approx(om, abs=1e-10)


def test_unbiased_over_the_phases():
    nx = ny = 6
    model, h, a, b = _cell(nx, ny)
    M = 64
    F1, _ = kpm.f_spectral(h, a, b, M)
    exact = kpm.observables(model, F1)
    one = probing.observables_probing(model, h, a, b, M, 2, seed=0)[0]
    mean = np.mean([probing.observables_probing(model, h, a, b, M, 2, seed=s)[0] for s in range(64)], axis=0)
    e1, em = np.max(np.abs(one - exact)), np.max(np.abs(mean - exact))
    assert e1 > 1e-4                  # one draw carries the contamination
    assert em < 0.35 * e1             # the average over 64 draws shrinks it (~1/8)


def test_error_falls_with_colour_spacing():
    nx = ny = 12
    model, h, a, b = _cell(nx, ny)
    M = 64
    F1, _ = kpm.f_spectral(h, a, b, M)
    exact = kpm.observables(model, F1)
    errs = [np.max(np.abs(probing.observables_probing(model, h, a, b, M, p, seed=1)[0] - exact))
            for p in (2, 3, 4, 6, 12)]
    assert errs[-1] < 1e-12
    assert errs[0] > errs[2] > errs[3] > errs[-1]


def test_recursion_route_equals_spectral_route():
    # the naive recursion on selected probing vectors reproduces the dense estimate
    nx = ny = 6
    model, h, a, b = _cell(nx, ny)
    M, p, seed = 48, 3, 7
    dense, _ = probing.f_probing(h, a, b, M, nx, ny, p, seed)
    fld_model = rmft.Model(nx, ny)
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64)
    from oracle import bdg as _bdg
    fld = rmft.fields(fld_model, inputs.vortex_seed(w), 0.3)
    J, F = probing.columns_probing_naive(_bdg.csr(fld_model, fld), a, b, M, nx, ny, p, seed, [0, 1, 7])
    assert len(J) == 3 * (nx // p) * (ny // p)
    assert np.max(np.abs(F - dense[:, J])) < 1e-12
