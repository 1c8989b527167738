"""Vortex-profile order parameters on the GPU (Eqs. giDelta, gm) against the
oracle, with and without magnetic order."""
import numpy as np
import pytest

from oracle import diagnostics, rmft
from paper_2212_05685_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["vortex", "random", "neel"])
def test_order_parameters_match_oracle(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_05685_gb300 import build, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    nx, ny = 12, 8
    N = nx * ny
    if case == "vortex":
        p = inputs.vortex_seed(inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64))
    elif case == "random":
        p = inputs.random_params(nx, ny, 6, spin_split=0.02)
    else:  # Neel order without bonds: every ratio R = X^2 > 0
        st = (-1.0) ** (np.arange(N) % nx + np.arange(N) // nx)
        n = np.stack([0.45 + 0.04 * st, 0.45 - 0.04 * st])
        p = rmft.join(n, np.zeros((2, 4, N), complex), np.zeros((4, N), complex))
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    d = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    mg = torch.empty(N, dtype=torch.float64, device="cuda")
    kpm.kpm_order_parameters(ctx, model, phi, torch.tensor(p, device="cuda"), d, mg)
    torch.cuda.synchronize()
    om = rmft.Model(nx, ny, phi=phi.cpu().numpy().reshape(4, N))
    dref = diagnostics.physical_pairing(om, p)
    mref = diagnostics.staggered_magnetisation(om, p)
    got = d.cpu().numpy().reshape(N, 2)
    assert np.max(np.abs(got[:, 0] + 1j * got[:, 1] - dref)) < 1e-13
    # the square root of g^z/g^xy is undefined where a bond ratio is negative
    # (random magnetic states): NaN on both sides there
    got_m = mg.cpu().numpy()
    assert np.array_equal(np.isnan(got_m), np.isnan(mref))
    ok = ~np.isnan(mref)
    if case != "random":
        assert ok.all()
    if ok.any():
        assert np.max(np.abs(got_m[ok] - mref[ok])) < 1e-12 * max(1.0, np.max(np.abs(mref[ok])))
    if case == "neel":
        assert np.min(np.abs(mref)) > 0.01
    if case == "vortex":
        assert np.max(np.abs(mref)) == 0.0
    kpm.kpm_destroy(ctx)
