"""Pins of the LDOS (App. C, Eqs. N_i, Gij; reading L1): the truncated
Chebyshev resolvent series against the Lorentzians of the eigenpairs, the
spectral sum rule, and the particle-hole relation of the two spin parts."""
import numpy as np
import pytest

from oracle import bdg, ldos, rmft
from paper_2212_05685_gb300 import inputs


def _cell(nx=6, ny=4, sym=False):
    model = rmft.Model(nx, ny)
    if sym:
        p = inputs.vortex_seed(inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64))
    else:
        p = inputs.random_params(nx, ny, 4)
    fld = rmft.fields(model, p, 0.2)
    h = bdg.dense(model, fld)
    a, b = bdg.gershgorin(model, fld)
    return model, p, h, a, b


def test_series_equals_lorentzians_at_wide_broadening():
    # |w|^M negligible: the truncated series is the exact resolvent
    model, p, h, a, b = _cell(sym=True)
    om = np.linspace(-1.5, 1.5, 13)
    ex = ldos.ldos_exact(h, om, alpha=0.0, gamma0=0.3)
    ch, _ = ldos.ldos_cheb(h, a, b, 600, om, alpha=0.0, gamma0=0.3)
    assert np.max(np.abs(ch - ex)) < 1e-11


def test_series_converges_with_M_at_the_paper_broadening():
    model, p, h, a, b = _cell(sym=True)
    om = np.array([-0.4, -0.05, 0.0, 0.1, 0.6])
    ex = ldos.ldos_exact(h, om, alpha=0.25, gamma0=0.02)
    errs = [np.max(np.abs(ldos.ldos_cheb(h, a, b, M, om, alpha=0.25, gamma0=0.02)[0] - ex))
            for M in (256, 1024, 4096)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def test_spectral_sum_rule():
    # each Nambu row's spectral function integrates to 1 (Lorentzians of fixed width)
    model, p, h, a, b = _cell()
    om = np.linspace(-60.0, 60.0, 240001)
    n = ldos.ldos_exact(h, om, alpha=0.0, gamma0=0.05)
    integral = np.trapezoid(n, om, axis=1)
    assert np.max(np.abs(integral - 1.0)) < 2e-3


def test_spin_parts_in_the_particle_hole_sector():
    # symmetric sector: the (i, dn) spectral function at -omega equals the
    # (i, up) one at omega (U conj(h) U^T = -h), so both spin parts agree
    model, p, h, a, b = _cell(sym=True)
    om = np.linspace(-1.0, 1.0, 9)
    n = ldos.ldos_exact(h, om, alpha=0.25, gamma0=0.01)
    assert np.max(np.abs(n[0] - n[1])) < 1e-10


def test_gutzwiller_weights_reduce_to_gt_squared():
    N = 6 * 4
    p = inputs.random_params(6, 4, 4)
    wgt = ldos.gutzwiller_weights(p, N)
    n, _, _ = rmft.split(p, N)
    d = 1 - n[0] - n[1]
    m = 0.5 * (n[0] - n[1])
    for s, sg in ((0, 1.0), (1, -1.0)):
        gt2 = 2 * d * (1 - d) / (1 - d * d + 4 * m * m) * (1 + d + 2 * sg * m) / (1 + d - 2 * sg * m)
        assert np.max(np.abs(wgt[s] - gt2)) < 1e-14
