"""Pins of the density-matrix routes of the oracle (App. B).

O1 (spectral KPM) and O2 (Chebyshev recursion on unit vectors) are two
independent evaluations of the same matrix polynomial; O0 is the exact
ground state.  Sum rules and the particle-hole structure of the Nambu matrix
fix further invariants.
"""
import numpy as np
import pytest

from oracle import bdg, kpm, rmft
from oracle.lattice import NN4
from paper_2212_05685_gb300 import inputs


def _setup(nx, ny, seed, flux=1, sym=False, mu=0.2):
    model = rmft.Model(nx, ny, flux=flux)
    if sym:
        p = inputs.vortex_seed(inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64, seed=seed))
    else:
        p = inputs.random_params(nx, ny, seed)
    fld = rmft.fields(model, p, mu)
    return model, p, fld


@pytest.mark.parametrize("nx,ny,M", [(4, 4, 64), (8, 8, 128), (5, 3, 40)])
def test_spectral_equals_recursion(nx, ny, M):
    model, _, fld = _setup(nx, ny, 3)
    h = bdg.dense(model, fld)
    a, b = bdg.gershgorin(model, fld)
    F1, om1 = kpm.f_spectral(h, a, b, M)
    F2, om2 = kpm.f_naive(bdg.csr(model, fld), a, b, M, block=37)
    assert np.max(np.abs(F1 - F2)) < 1e-11
    assert om1 == pytest.approx(om2, rel=1e-12, abs=1e-11)


def test_gershgorin_contains_spectrum_and_hermitian():
    model, _, fld = _setup(6, 5, 9)
    h = bdg.dense(model, fld)
    assert np.max(np.abs(h - h.conj().T)) == 0.0
    a, b = bdg.gershgorin(model, fld)
    E = np.linalg.eigvalsh(h)
    assert E.min() > b - a and E.max() < b + a
    # rows carry at most 13 entries (1 diagonal + 8 hops + 4 pairs)
    assert max(np.count_nonzero(r) for r in h) <= 13


def test_trace_moments_sum_rule():
    # mu_m = Tr T_m(h~): recursion traces equal sum_n T_m(x_n) (zeroth = D)
    model, _, fld = _setup(4, 4, 5)
    h = bdg.dense(model, fld)
    a, b = bdg.gershgorin(model, fld)
    D = h.shape[0]
    ht = (h - b * np.eye(D)) / a
    x = np.linalg.eigvalsh(ht)
    T0, T1 = np.eye(D), ht.copy()
    assert np.trace(T0).real == D
    assert np.trace(T1).real == pytest.approx(np.sum(x), abs=1e-11 * D)
    for m in range(2, 40):
        T0, T1 = T1, 2 * ht @ T1 - T0
        assert np.trace(T1).real == pytest.approx(np.sum(np.cos(m * np.arccos(np.clip(x, -1, 1)))), abs=1e-11 * D)


def test_particle_hole_symmetric_sector():
    # m = 0, equal spins and singlet pairing: E_n = -E_{D-1-n}, b = 0 and the
    # KPM density matrix keeps n_up = n_dn and sum_I rho_II = N exactly
    model, p, fld = _setup(8, 8, 0, sym=True)
    h = bdg.dense(model, fld)
    E = np.linalg.eigvalsh(h)
    assert np.max(np.abs(E + E[::-1])) < 1e-12
    a, b = bdg.gershgorin(model, fld)
    assert abs(b) < 1e-15
    F1, _ = kpm.f_spectral(h, a, b, 128)
    assert np.trace(F1).real == pytest.approx(model.N, abs=1e-10)
    o = kpm.observables(model, F1)
    n, chi, F = rmft.split(o, model.N)
    assert np.max(np.abs(n[0] - n[1])) < 1e-12
    assert np.max(np.abs(chi[0] - chi[1])) < 1e-12
    for e in range(4):  # F_{i,i+e} = F_{i+e,i}
        j = model.nn4[e]
        assert np.max(np.abs(F[e] - F[(e + 2) % 4][j])) < 1e-12


def test_particle_hole_half_relations():
    """What the particle-hole half pass relies on: in the symmetric sector
    (b = 0) the damped step series obeys F_M(h~) = 1 - U conj(F_M(h~)) U^T, i.e.
    entry ((k,dn),(j,dn)) = delta_kj - conj(entry ((k,up),(j,up))), and the
    grand potential's (j,dn) diagonal equals the (j,up) diagonal of G_M(-h~)."""
    model, p, fld = _setup(6, 5, 0, sym=True)
    h = bdg.dense(model, fld)
    a, b = bdg.gershgorin(model, fld)
    M = 96
    F1, _ = kpm.f_spectral(h, a, b, M)
    up, dn = np.arange(0, h.shape[0], 2), np.arange(1, h.shape[0], 2)
    lhs = F1[np.ix_(dn, dn)]
    rhs = np.eye(model.N) - np.conj(F1[np.ix_(up, up)])
    assert np.max(np.abs(lhs - rhs)) < 1e-12
    # F_M((k,up),(j,dn)) = conj(F_M((k,dn),(j,up))) elementwise
    assert np.max(np.abs(F1[np.ix_(up, dn)] - np.conj(F1[np.ix_(dn, up)]))) < 1e-12
    E, U = np.linalg.eigh(h)
    x = (E - b) / a
    _, ao = kpm.coefficients(M, a, b)
    w = np.abs(U) ** 2
    g_dn = w[dn] @ kpm.cheb_eval(ao, x)
    g_up_reflected = w[up] @ kpm.cheb_eval(ao, -x)
    assert np.max(np.abs(g_dn - g_up_reflected)) < 1e-12
    # so the sum over the (j,dn) diagonals uses the coefficients (-1)^m a^Omega_m
    signs = (-1.0) ** np.arange(M)
    assert np.max(np.abs(g_dn - w[up] @ kpm.cheb_eval(signs * ao, x))) < 1e-12


def test_kpm_converges_to_ground_state_with_M():
    # a gapped uniform d-wave state: exponential convergence of F_M to theta
    model = rmft.Model(12, 12, flux=0)
    p = inputs.uniform_dwave(12, 12, 0.1, pair=0.3)
    fld = rmft.fields(model, p, 0.0)
    h = bdg.dense(model, fld)
    a, b = bdg.gershgorin(model, fld)
    F0, om0 = kpm.f_ed(h)
    errs = []
    for M in (32, 64, 128, 256, 512):
        F1, om1 = kpm.f_spectral(h, a, b, M)
        errs.append(np.max(np.abs(F1 - F0)))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * errs[0]


def test_observable_extraction_uses_both_column_kinds():
    # the two Nambu columns give redundant copies of the pairing:
    # f[(j+e, 0), (j, 1)] = -F_{j+e, j} (column (j,1)) must equal the
    # column-(j+e, 0) value, by Hermiticity of f(h)
    model, _, fld = _setup(5, 4, 11)
    h = bdg.dense(model, fld)
    a, b = bdg.gershgorin(model, fld)
    F1, _ = kpm.f_spectral(h, a, b, 64)
    o = kpm.observables(model, F1)
    _, _, F = rmft.split(o, model.N)
    i = np.arange(model.N)
    for e in range(4):
        j = model.nn4[e]
        assert np.max(np.abs(F1[2 * j, 2 * i + 1] + F[(e + 2) % 4][j])) < 1e-13


def test_observables_at_sites_equals_full_readout():
    """The per-site readout from a few columns equals the full-matrix readout."""
    from oracle import bdg, kpm as okpm, rmft
    from paper_2212_05685_gb300 import inputs
    nx, ny, M = 6, 5, 40
    om = rmft.Model(nx, ny)
    f = rmft.fields(om, inputs.random_params(nx, ny, 12), 0.2)
    a, b = bdg.gershgorin(om, f)
    F1, _ = okpm.f_spectral(bdg.dense(om, f), a, b, M)
    ref = okpm.observables(om, F1)
    sites = np.array([0, 7, 29, 13])
    cols = np.sort(np.concatenate([2 * sites, 2 * sites + 1]))
    n, chi, F = okpm.observables_at(om, F1[:, cols], cols, sites)
    rn, rc, rF = rmft.split(ref, om.N)
    assert np.array_equal(n, rn[:, sites])
    assert np.array_equal(chi, rc[:, :, sites])
    assert np.array_equal(F, rF[:, sites])
