"""Many-body brute force pins of the Nambu conventions and Wick decomposition.

The Fock-space ground state of H_eff = sum h_IJ d^dag_I d_J is found by
Lanczos on the full 4^L space; correlations come straight from the state.
"""
import numpy as np
import pytest

from oracle import bdg, fock, kpm, rmft
from oracle.lattice import NN4
from paper_2212_05685_gb300 import inputs


@pytest.fixture(scope="module")
def cluster():
    return fock.Cluster(6)


@pytest.mark.parametrize("seed", [1, 2])
def test_density_matrix_is_transpose_of_f(cluster, seed):
    model = rmft.Model(3, 2)
    fld = rmft.fields(model, inputs.random_params(3, 2, seed, spin_split=0.03), 0.1 * seed)
    h = bdg.dense(model, fld)
    psi, w = cluster.ground_state(h)
    assert w[1] - w[0] > 1e-6  # non-degenerate ground state
    rho = cluster.rho_nambu(psi)
    F0, _ = kpm.f_ed(h)
    # rho_IJ = <d^dag_I d_J> = f(h)_JI  (reading N1)
    assert np.max(np.abs(rho - F0.T)) < 1e-10


@pytest.mark.parametrize("seed", [3, 4])
def test_observables_match_many_body_correlators(cluster, seed):
    model = rmft.Model(3, 2)
    fld = rmft.fields(model, inputs.random_params(3, 2, seed, spin_split=-0.02), -0.1)
    h = bdg.dense(model, fld)
    psi, _ = cluster.ground_state(h)
    F0, _ = kpm.f_ed(h)
    n, chi, F = rmft.split(kpm.observables(model, F0), model.N)
    for i in range(model.N):
        for s in range(2):
            assert n[s, i] == pytest.approx(cluster.hop(psi, i, i, s).real, abs=1e-10)
        for d in range(4):
            j = model.fwd[d][i]
            if j == i:
                continue
            for s in range(2):
                # on the 3 x 2 torus two bonds may join the same pair; chi is the
                # single correlator <c^dag_i c_j> either way
                assert chi[s, d, i] == pytest.approx(cluster.hop(psi, i, j, s), abs=1e-10)
        for e in range(4):
            j = model.nn4[e][i]
            assert F[e, i] == pytest.approx(cluster.pair(psi, i, j), abs=1e-10)


def test_wick_exchange_terms(cluster):
    # W2: <S^z_i S^z_j> = m_i m_j - 1/4 sum_s(|chi_s|^2 + |Delta_s|^2),
    #     <(S+S- + S-S+)/2> = -Re(chi_up chi_dn^* + Delta_up^* Delta_dn)
    model = rmft.Model(3, 2)
    fld = rmft.fields(model, inputs.random_params(3, 2, 7, spin_split=0.04, scale=2.0), 0.05)
    h = bdg.dense(model, fld)
    psi, _ = cluster.ground_state(h)
    F0, _ = kpm.f_ed(h)
    n, chi, F = rmft.split(kpm.observables(model, F0), model.N)
    m = 0.5 * (n[0] - n[1])
    for i in range(model.N):
        j = model.fwd[0][i]      # +x bond
        Fij = F[0, i]
        Fji = F[2, j]
        szz, sxy = cluster.spin_corr(psi, i, j)
        cu, cd = chi[0, 0, i], chi[1, 0, i]
        ref_zz = m[i] * m[j] - 0.25 * (abs(cu) ** 2 + abs(cd) ** 2 + abs(Fij) ** 2 + abs(Fji) ** 2)
        ref_xy = -(cu * np.conj(cd) + np.conj(Fij) * Fji).real
        assert szz == pytest.approx(ref_zz, abs=1e-10)
        assert sxy == pytest.approx(ref_xy, abs=1e-10)
