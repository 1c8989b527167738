"""Finite temperature on the GPU (App. B, Eq. F_KPM at T > 0; coefficients by
Chebyshev-Gauss quadrature) against the oracle: full, particle-hole half and
probing passes, FP64 <= 1e-10 and FP32 <= 2e-5."""
import numpy as np
import pytest

from oracle import bdg, kpm as okpm, probing, rmft
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


def _setup(K, nx, ny, p, mu):
    kpm, ctx = K
    N = nx * ny
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, torch.tensor(p, device="cuda"), mu, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    return model, fields, ab


def _gpu(K, model, fields, ab, opts):
    kpm, ctx = K
    N = model.nx * model.ny
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    om = torch.empty(1, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, opts, fields, ab, obs, om)
    torch.cuda.synchronize()
    return obs.cpu().numpy(), float(om.item())


@pytest.mark.parametrize("T", [0.02, 0.1, 0.5])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_finite_temperature_pass(K, T, prec):
    kpm, _ = K
    nx, ny, M = 10, 8, 96
    model, fields, ab = _setup(K, nx, ny, inputs.random_params(nx, ny, 3), 0.2)
    P = kpm.KPM_FP64 if prec == "fp64" else kpm.KPM_FP32
    got, om = _gpu(K, model, fields, ab, kpm.make_opts(M, P, temperature=T))
    o = rmft.Model(nx, ny)
    a, b = ab.cpu().numpy()
    F1, omega = okpm.f_spectral(bdg.dense(o, fields.cpu().numpy()), a, b, M, T)
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.max(np.abs(got - okpm.observables(o, F1))) < tol
    assert om == pytest.approx(omega, rel=1e-10 if prec == "fp64" else 1e-5)


def test_finite_temperature_half_and_probing(K):
    kpm, _ = K
    nx, ny, M, T = 12, 12, 80, 0.05
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M)
    model, fields, ab = _setup(K, nx, ny, inputs.vortex_seed(w), 0.3)
    full, om = _gpu(K, model, fields, ab, kpm.make_opts(M, kpm.KPM_FP64, temperature=T))
    half, om_h = _gpu(K, model, fields, ab, kpm.make_opts(M, kpm.KPM_FP64, temperature=T,
                                                          flags=kpm.KPM_FLAG_PH_HALF))
    assert np.max(np.abs(half - full)) < 1e-10
    assert om_h == pytest.approx(om, rel=1e-11)
    est, om_p = _gpu(K, model, fields, ab, kpm.make_opts(M, kpm.KPM_FP64, temperature=T, probe_p=3, probe_seed=2))
    o = rmft.Model(nx, ny)
    a, b = ab.cpu().numpy()
    ref, omega = probing.observables_probing(o, bdg.dense(o, fields.cpu().numpy()), a, b, M, 3, 2, T)
    assert np.max(np.abs(est - ref)) < 1e-10
    assert om_p == pytest.approx(omega, rel=1e-10)


def test_negative_temperature_is_refused(K):
    kpm, _ = K
    model, fields, ab = _setup(K, 6, 4, inputs.random_params(6, 4, 1), 0.0)
    with pytest.raises(kpm.KPMError):
        _gpu(K, model, fields, ab, kpm.make_opts(16, kpm.KPM_FP64, temperature=-0.1))
