"""Gauge covariance of the CUDA path (Sec. II): a site gauge transformation of
the Peierls phases and order parameters transforms every observable the same
way and leaves Omega unchanged (larger lattices than the oracle pins)."""
import math

import numpy as np
import pytest

from oracle import rmft
from paper_2212_05685_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gauge(nx, ny, theta, phi, p):
    model = rmft.Model(nx, ny, flux=0)
    N = nx * ny
    n, chi, F = rmft.split(p, N)
    phi2 = np.array(phi, dtype=np.float64, copy=True).reshape(4, N)
    chi2, F2 = chi.copy(), F.copy()
    for d in range(4):
        j = model.fwd[d]
        phi2[d] = phi2[d] + theta - theta[j]
        chi2[:, d] = chi[:, d] * np.exp(1j * (theta[j] - theta))
    for e in range(4):
        j = model.nn4[e]
        F2[e] = F[e] * np.exp(1j * (theta + theta[j]))
    return phi2.reshape(-1), rmft.join(n, chi2, F2)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_gauge_covariance_on_the_gpu(prec, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_05685_gb300 import build, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    nx, ny, M = 32, 16, 96
    N = nx * ny
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p = inputs.random_params(nx, ny, 5)
    theta = np.random.default_rng(9).uniform(-math.pi, math.pi, size=N)
    phi2, p2 = _gauge(nx, ny, theta, phi.cpu().numpy(), p)
    P = kpm.KPM_FP64 if prec == "fp64" else kpm.KPM_FP32

    def run(ph, pp):
        f = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        kpm.kpm_build_H(ctx, model, torch.tensor(ph, device="cuda"), torch.tensor(pp, device="cuda"), 0.2, f)
        ab = torch.empty(2, dtype=torch.float64, device="cuda")
        kpm.kpm_bounds(ctx, model, f, 0.01, ab)
        obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        om = torch.empty(1, dtype=torch.float64, device="cuda")
        kpm.kpm_observables(ctx, model, kpm.make_opts(M, P), f, ab, obs, om)
        torch.cuda.synchronize()
        return obs.cpu().numpy(), float(om.item())

    o, om = run(phi.cpu().numpy(), p)
    o2, om2 = run(phi2, p2)
    _, expect = _gauge(nx, ny, theta, phi.cpu().numpy(), o)
    assert np.max(np.abs(o2 - expect)) < tol
    assert om2 == pytest.approx(om, rel=1e-10 if prec == "fp64" else 1e-5)
    kpm.kpm_destroy(ctx)
