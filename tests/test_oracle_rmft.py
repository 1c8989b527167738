"""Pins of the RMFT functional and its effective fields (App. A).

The analytic fields are checked against central differences of W; the
Gutzwiller factors against their closed m = 0 forms; the Nambu assembly
against the linearisation of W (h_IJ = dW/drho_IJ); the self-consistency
loop against the uniform solution it must reach.
"""
import numpy as np
import pytest

from oracle import bdg, kpm, kspace, rmft
from paper_2212_05685_gb300 import inputs


def _fd(fun, p, k, h=1e-5):
    # fourth-order central difference
    def at(s):
        q = p.copy()
        q[k] += s
        return fun(q)
    return (8 * (at(h) - at(-h)) - (at(2 * h) - at(-2 * h))) / (12 * h)


@pytest.mark.parametrize("gutz,split", [(True, 0.0), (True, 0.03), (False, 0.02)])
def test_fields_are_derivatives_of_W(gutz, split):
    nx, ny = 4, 3
    N = nx * ny
    model = rmft.Model(nx, ny, gutzwiller=gutz)
    p = inputs.random_params(nx, ny, 5, spin_split=split)
    mu = 0.37
    f = rmft.fields(model, p, mu)
    W = lambda q: rmft.energy_W(model, q, mu, 0.875)
    rng = np.random.default_rng(1)
    # eps = dW/dn
    for k in rng.choice(2 * N, 8, replace=False):
        assert f[k] == pytest.approx(_fd(W, p, k), abs=2e-9)
    # T = dW/dchi = (dW/dRe - i dW/dIm)/2 ; D = dW/dF* = (dW/dRe + i dW/dIm)/2
    for off, n_c, conj in ((2 * N, 8 * N, -1.0), (18 * N, 4 * N, 1.0)):
        for c in rng.choice(n_c, 10, replace=False):
            k = off + 2 * c
            num = 0.5 * (_fd(W, p, k) + conj * 1j * _fd(W, p, k + 1))
            assert complex(f[k], f[k + 1]) == pytest.approx(num, abs=2e-9)


def test_gutzwiller_factors_reduce_at_m_zero():
    # m = 0: g^t_ij = 2 delta/(1 + delta) and g^xy_ij = 4/(1 + delta)^2 for
    # uniform delta; g^z = g^xy
    for delta in (0.05, 0.125, 0.3):
        n = np.full((2, 3), 0.5 * (1 - delta))
        sf = rmft.site_factors(n)
        assert sf["gt"][0, 0] ** 2 == pytest.approx(2 * delta / (1 + delta), rel=1e-14)
        assert sf["gt"][1, 0] ** 2 == pytest.approx(2 * delta / (1 + delta), rel=1e-14)
        assert sf["gxy"][0] ** 2 == pytest.approx(4 / (1 + delta) ** 2, rel=1e-14)
    R, dA, dc, dX = rmft._ratio(np.array([-0.04, 0.1]), np.array([0.0, 0.0]), np.array([10.0, 3.0]))
    assert np.all(R == 1.0) and np.all(dA == 0.0) and np.all(dX == 0.0)


def test_site_factor_derivatives_match_differences():
    rng = np.random.default_rng(3)
    n = 0.42 + 0.05 * rng.uniform(-1, 1, size=(2, 5))
    sf = rmft.site_factors(n)
    h = 1e-6
    for sp in range(2):
        npl, nmi = n.copy(), n.copy()
        npl[sp] += h
        nmi[sp] -= h
        a, b = rmft.site_factors(npl), rmft.site_factors(nmi)
        for s in range(2):
            assert np.max(np.abs((a["gt"][s] - b["gt"][s]) / (2 * h) - sf["dgt"][s, sp])) < 1e-8
        assert np.max(np.abs((a["gxy"] - b["gxy"]) / (2 * h) - sf["dgxy"][sp])) < 1e-8


def test_nambu_matrix_is_gradient_of_W():
    # sum_IJ h_IJ rho_IJ = sum_fields dW/dO * O - sum_i eps_{i dn}: the Nambu
    # matrix built from the fields is the gradient of W in rho, so its ground
    # state minimises the linearised W (variational principle of App. A)
    model = rmft.Model(4, 4)
    N = model.N
    p = inputs.random_params(4, 4, 3, spin_split=0.02)
    f = rmft.fields(model, p, 0.3)
    h = bdg.dense(model, f)
    eps, T, D = rmft.split(f, N)
    for seed in range(3):
        h0 = bdg.dense(model, rmft.fields(model, inputs.random_params(4, 4, 10 + seed), 0.1 * seed))
        F0, _ = kpm.f_ed(h0)
        n, chi, Fo = rmft.split(kpm.observables(model, F0), N)
        Elin = np.trace(h @ F0).real
        Wlin = np.sum(eps * n) + 2 * np.sum((T * chi).real) + 2 * np.sum((np.conj(D) * Fo).real)
        assert Elin - Wlin == pytest.approx(-np.sum(eps[1]), abs=1e-10)


def test_uniform_loop_reaches_momentum_space_fixed_point():
    # zero field, uniform d-wave seed: the loop converges to a uniform state,
    # and that state is a fixed point of the momentum-space KPM map at the
    # same order M (independent of the real-space recursion)
    nx = ny = 8
    M, nt = 96, 0.875
    model = rmft.Model(nx, ny, flux=0)
    p = inputs.uniform_dwave(nx, ny, 1 - nt)
    mu_eff = 0.0
    for it in range(200):
        f, mu = rmft.shifted_fields(model, p, mu_eff)
        h = bdg.dense(model, f)
        a, b = bdg.gershgorin(model, f)
        F1, _ = kpm.f_spectral(h, a, b, M)
        p, mu_eff, r, e = rmft.update(p, kpm.observables(model, F1), nt, mu_eff)
        if r < 1e-10 and abs(e) < 1e-10:
            break
    assert r < 1e-10 and abs(e) < 1e-10
    f, mu = rmft.shifted_fields(model, p, mu_eff)
    a, b = bdg.gershgorin(model, f)
    ok, _ = kspace.kpm_uniform(nx, ny, kspace.site_fields(f, model.N), a, b, M)
    assert np.max(np.abs(ok - p)) < 1e-9
    n, chi, F = rmft.split(p, model.N)
    assert abs(F[0, 0]) > 0.05 and F[0, 0].real * F[1, 0].real < 0   # d-wave survives
    # the variational energy is below that of the normal state at equal chi
    pn = p.copy()
    pn[18 * model.N:] = 0.0
    assert rmft.energy_W(model, p, mu, nt) < rmft.energy_W(model, pn, mu, nt)


def test_update_rule():
    N = 3
    p = np.zeros(26 * N)
    o = np.arange(26 * N, dtype=float) * 0.01
    new, mu, r, e = rmft.update(p, o, 0.0, 1.0, alpha=0.5, alpha_n=0.1, eta=0.5, paramagnetic=True)
    avg = 0.5 * (o[:N] + o[N:2 * N])
    e_ref = 2 * np.sum(avg) / N
    assert e == pytest.approx(e_ref)
    assert mu == pytest.approx(1.0 - 0.5 * e_ref)
    assert np.allclose(new[:N], 0.1 * (avg - 0.5 * e_ref))
    assert np.allclose(new[2 * N:], 0.5 * o[2 * N:])
    assert r == pytest.approx(np.max(np.abs(o[2 * N:])))
