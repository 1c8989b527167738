"""Pins of the reverse-mode gradients (App. B, Eqs. dFdH, dalphadH).

The backward recursion is checked against finite differences of the forward
KPM pass (rescaling held fixed), against the Daleckii-Krein derivative of the
matrix polynomial, and against the Hellmann-Feynman closed form: the
gradient of the ground-state grand potential with respect to the Nambu
matrix is the density matrix, so dOmega/d(eps, T, D) are the observables.
"""
import numpy as np
import pytest

from oracle import adjoint, bdg, kpm, rmft
from paper_2212_05685_gb300 import inputs


def _setup(nx, ny, seed, mu=0.2, flux=1):
    model = rmft.Model(nx, ny, flux=flux)
    p = inputs.random_params(nx, ny, seed)
    fld = rmft.fields(model, p, mu)
    a, b = bdg.gershgorin(model, fld)
    return model, p, fld, a, b


def _random_upstream(N, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=26 * N), float(rng.normal())


def _loss_at(model, fld, a, b, M, g_obs, g_om):
    F1, om = kpm.f_spectral(bdg.dense(model, fld), a, b, M)
    return adjoint.loss(model, kpm.observables(model, F1), g_obs, om, g_om)


def test_vjp_matches_finite_differences():
    model, _, fld, a, b = _setup(4, 3, 2)
    M = 40
    g_obs, g_om = _random_upstream(model.N, 7)
    grad = adjoint.vjp_dense(model, fld, a, b, M, g_obs, g_om)
    rng = np.random.default_rng(1)
    h = 1e-3

    def at(k, s):
        f = fld.copy()
        f[k] += s
        return _loss_at(model, f, a, b, M, g_obs, g_om)

    for k in rng.choice(26 * model.N, 25, replace=False):
        # fourth-order central difference (the loss is a polynomial in h~)
        fd = (8 * (at(k, h) - at(k, -h)) - (at(k, 2 * h) - at(k, -2 * h))) / (12 * h)
        # real layout: component k of the gradient is dL/d(component k)
        assert grad[k] == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_recursion_equals_daleckii_krein():
    model, _, fld, a, b = _setup(5, 3, 4)
    M = 33
    g_obs, g_om = _random_upstream(model.N, 3)
    g1 = adjoint.vjp_dense(model, fld, a, b, M, g_obs, g_om)
    g2 = adjoint.vjp_recursion(model, fld, a, b, M, g_obs, g_om)
    assert np.max(np.abs(g1 - g2)) < 1e-11 * max(1.0, np.max(np.abs(g1)))


def test_hellmann_feynman_limit():
    # gapped uniform d-wave state: dOmega_M/dfields -> the ED observables
    model = rmft.Model(8, 8, flux=0)
    p = inputs.uniform_dwave(8, 8, 0.1, pair=0.3)
    fld = rmft.fields(model, p, 0.0)
    a, b = bdg.gershgorin(model, fld)
    h = bdg.dense(model, fld)
    F0, _ = kpm.f_ed(h)
    hf = adjoint.field_grad_from_G(model, F0, 1.0)
    # closed forms of the Hellmann-Feynman gradient in the field layout
    obs = kpm.observables(model, F0)
    n, chi, F = rmft.split(obs, model.N)
    e_hf, T_hf, D_hf = rmft.split(hf, model.N)
    assert np.max(np.abs(e_hf[0] - n[0])) < 1e-12
    assert np.max(np.abs(e_hf[1] - (n[1] - 1.0))) < 1e-12
    assert np.max(np.abs(T_hf - 2 * np.conj(chi))) < 1e-12
    assert np.max(np.abs(D_hf - 2 * np.conj(F))) < 1e-12
    zero = np.zeros(26 * model.N)
    errs = []
    for M in (64, 128, 256, 512):
        g = adjoint.vjp_dense(model, fld, a, b, M, zero, 1.0)
        errs.append(np.max(np.abs(g - hf)))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-4


def test_phase_gradient_matches_finite_differences():
    nx, ny = 4, 3
    p = inputs.random_params(nx, ny, 6)
    base = rmft.Model(nx, ny)
    g_fields = np.random.default_rng(2).normal(size=26 * base.N)
    gphi = adjoint.phi_grad(base, p, g_fields)

    def L(phi):
        m = rmft.Model(nx, ny, phi=phi)
        return float(np.sum(g_fields * rmft.fields(m, p, 0.3)))

    h = 1e-6
    for k in range(0, 4 * base.N, 5):
        pp, pm = base.phi.copy().reshape(-1), base.phi.copy().reshape(-1)
        pp[k] += h
        pm[k] -= h
        fd = (L(pp.reshape(4, -1)) - L(pm.reshape(4, -1))) / (2 * h)
        assert gphi[k] == pytest.approx(fd, rel=1e-6, abs=1e-8)
