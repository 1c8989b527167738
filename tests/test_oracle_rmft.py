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


# ---------------------------------------------------------------- magnetic points (m != 0)
# Values of App. A's Gutzwiller factors worked out by hand (exact fractions)
# at two magnetic points, written here as literals with their derivation.
#
# Point A: n_up = 1/2, n_dn = 3/10 -> delta = 1/5, m = 1/10, P = 1 - delta^2 + 4 m^2 = 1
#   g^t_up^2 = 2 delta (1 - delta)/P * (1 + delta + 2m)/(1 + delta - 2m) = (8/25)(7/5) = 56/125
#   g^t_dn^2 = (8/25)(1/(7/5))                                            = 8/35
#   g^xy     = 2 (1 - delta)/P                                            = 8/5
# Point B: n_up = 9/20, n_dn = 2/5 -> delta = 3/20, m = 1/40, P = 1 - 9/400 + 1/400 = 49/50
#   g^t_up^2 = (2 (3/20)(17/20)/(49/50)) (6/5)/(11/10) = (51/196)(12/11)  = 153/539
#   g^t_dn^2 = (51/196)(11/12)                                           = 187/784
#   g^xy     = (17/10)/(49/50)                                           = 85/49
from fractions import Fraction as Fr  # noqa: E402


def _magnetic_params(nx, ny, dens, chi=None, F=None):
    N = nx * ny
    n = np.zeros((2, N))
    n[0], n[1] = 0.45, 0.45
    for i, (nu, nd) in dens.items():
        n[0, i], n[1, i] = nu, nd
    c = np.zeros((2, 4, N), dtype=np.complex128)
    f = np.zeros((4, N), dtype=np.complex128)
    for (s, d, i), v in (chi or {}).items():
        c[s, d, i] = v
    for (e, i), v in (F or {}).items():
        f[e, i] = v
    return inputs.pack(n, c, f)


@pytest.mark.parametrize("nu,nd,gt_up2,gt_dn2,gxy", [
    (Fr(1, 2), Fr(3, 10), Fr(56, 125), Fr(8, 35), Fr(8, 5)),
    (Fr(9, 20), Fr(2, 5), Fr(153, 539), Fr(187, 784), Fr(85, 49)),
])
def test_gutzwiller_site_factors_at_magnetic_points(nu, nd, gt_up2, gt_dn2, gxy):
    n = np.array([[float(nu)], [float(nd)]])
    sf = rmft.site_factors(n)
    assert sf["gt"][0, 0] == pytest.approx(float(gt_up2) ** 0.5, rel=1e-14)
    assert sf["gt"][1, 0] == pytest.approx(float(gt_dn2) ** 0.5, rel=1e-14)
    assert sf["gxy"][0] == pytest.approx(float(gxy), rel=1e-14)


def test_gsz_and_X_of_a_magnetic_bond():
    """One x bond i -> j with m_i = 1/10, m_j = -1/10 (point A and its mirror
    n_up <-> n_dn, both delta = 1/5, P = 1), chi_up = 3/10, chi_dn = 1/10
    (chibar = 1/5), Delta_up = F_ij = 2/5, Delta_dn = F_ji = 1/5 (Deltabar = 3/10):
      X = 1 + 12 (4/5)(4/5)/sqrt(1 * 1) = 217/25
      A = 2 (|Deltabar|^2 - |chibar|^2) = 2 (9/100 - 4/100) = 1/10
      c = 4 m_i m_j = -1/25
      R = (A - c X^2)/(A - c) = (1/10 + 47089/15625)/(7/50) = 97303/4375
      g^xy_ij = (8/5)(8/5) = 64/25,  g^z_ij = (64/25)(97303/4375)
    and the bond's exchange energy (reading W2)
      J [g^z (m_i m_j - (|chi_up|^2 + |chi_dn|^2 + |D_up|^2 + |D_dn|^2)/4)
         - g^xy Re(chi_up chi_dn* + D_up* D_dn)]
      = J [g^z (-1/100 - 3/40) - (64/25)(3/100 + 2/25)]."""
    nx, ny = 4, 2
    om = rmft.Model(nx, ny, flux=0)
    i, j = 0, 1
    p = _magnetic_params(nx, ny, {i: (0.5, 0.3), j: (0.3, 0.5)},
                         chi={(0, 0, i): 0.3, (1, 0, i): 0.1},
                         F={(0, i): 0.4, (2, j): 0.2})
    n, chi, F = rmft.split(p, om.N)
    sf = rmft.site_factors(n)
    b = rmft._bond_exchange(om, sf, n, chi, F, 0)
    X = Fr(217, 25)
    R = Fr(97303, 4375)
    gz = Fr(64, 25) * R
    assert b["X"][i] == pytest.approx(float(X), rel=1e-14)
    assert b["R"][i] == pytest.approx(float(R), rel=1e-13)
    assert b["gz"][i] == pytest.approx(float(gz), rel=1e-13)
    Ebond = om.J * (float(gz) * (-0.01 - 0.075) - 2.56 * (0.03 + 0.08))
    assert b["W"][i] == pytest.approx(Ebond, rel=1e-13)


def test_W_of_a_magnetic_bond_configuration():
    """W of the configuration above (zero field, only the bond i -> j carries
    chi and F, every other site paramagnetic so no other bond has m_i m_j != 0):
      hopping  -2 t (g^t_i,up g^t_j,up chi_up + g^t_i,dn g^t_j,dn chi_dn)
               with g^t_j,up = g^t_i,dn and g^t_j,dn = g^t_i,up (mirror point),
               g^t_i,up g^t_j,up = sqrt((56/125)(8/35)) = sqrt(64/625) = 8/25:
               -2 (8/25)(3/10 + 1/10) = -32/125
      exchange the bond energy of the previous test
      mu term  0 (mu = 0)."""
    nx, ny = 4, 2
    om = rmft.Model(nx, ny, flux=0)
    p = _magnetic_params(nx, ny, {0: (0.5, 0.3), 1: (0.3, 0.5)},
                         chi={(0, 0, 0): 0.3, (1, 0, 0): 0.1}, F={(0, 0): 0.4, (2, 1): 0.2})
    gz = float(Fr(64, 25) * Fr(97303, 4375))
    hop = -32.0 / 125.0
    exch = om.J * (gz * (-0.01 - 0.075) - 2.56 * (0.03 + 0.08))
    assert rmft.energy_W(om, p, 0.0) == pytest.approx(hop + exch, rel=1e-13)
