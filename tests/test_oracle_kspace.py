"""The momentum-space route against the real-space spectral KPM (zero field)."""
import numpy as np
import pytest

from oracle import bdg, kpm, kspace, rmft
from paper_2212_05685_gb300 import inputs


@pytest.mark.parametrize("nx,ny,M", [(8, 8, 64), (6, 10, 200)])
def test_kspace_matches_real_space(nx, ny, M):
    model = rmft.Model(nx, ny, flux=0)
    p = inputs.uniform_dwave(nx, ny, 0.14, chi_nn=0.18 + 0.02j, chi_nnn=-0.03, pair=0.09)
    f = rmft.fields(model, p, 1.7)
    h = bdg.dense(model, f)
    a, b = bdg.gershgorin(model, f)
    F1, om1 = kpm.f_spectral(h, a, b, M)
    o1 = kpm.observables(model, F1)
    ok, omk = kspace.kpm_uniform(nx, ny, kspace.site_fields(f, model.N), a, b, M)
    assert np.max(np.abs(ok - o1)) < 1e-12
    assert omk == pytest.approx(om1, rel=1e-12)
