"""kpm_opts.band_rows (lattice rows per CTA of the one-step recursion
kernels) changes the launch shape only: every band height gives the same bits
as the library's default, for FP32 (TMA-staged and cp.async chunks), FP64,
the half pass and the probing estimator, on lattices with ragged last bands;
a negative height is refused."""
import numpy as np
import pytest

from paper_2212_05685_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_05685_gb300 import build, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    yield kpm, ctx
    kpm.kpm_destroy(ctx)


def _pass(K, nx, ny, M, prec, band, cols=0, flags=0, probe_p=0):
    kpm, ctx = K
    N = nx * ny
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    if flags & kpm.KPM_FLAG_PH_HALF:
        ab[1] = 0.0
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    om = torch.zeros(1, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, kpm.make_opts(M, prec, 0, cols, flags=flags, probe_p=probe_p, probe_seed=3,
                                                  band_rows=band), fields, ab, obs, om)
    torch.cuda.synchronize()
    return obs.cpu().numpy(), float(om.item())


@pytest.mark.parametrize("nx,ny,M,prec,cols,flags,probe_p", [
    (24, 12, 33, 1, 16, 0, 0),      # FP32, TMA-staged chunks
    (20, 13, 20, 1, 4, 0, 0),       # FP32, cp.async chunks, odd ny
    (48, 24, 17, 1, 0, 2, 0),       # half pass
    (20, 12, 25, 1, 0, 0, 4),       # probing, R = 32
    (12, 10, 16, 0, 0, 0, 0),       # FP64
])
def test_band_rows_give_the_same_bits(K, nx, ny, M, prec, cols, flags, probe_p):
    ref, om_ref = _pass(K, nx, ny, M, prec, 0, cols, flags, probe_p)
    for band in (1, 2, 3, 5, ny - 1, ny, ny + 7):
        got, om = _pass(K, nx, ny, M, prec, band, cols, flags, probe_p)
        assert np.array_equal(ref, got), band
        assert om == om_ref, band


def test_negative_band_rows_refused(K):
    kpm, ctx = K
    with pytest.raises(kpm.KPMError) as e:
        _pass(K, 8, 8, 8, 1, -1)
    assert e.value.status == kpm.KPM_EINVAL
