"""LDOS on the GPU (App. C, Eqs. N_i, Gij; reading L1) against the oracle's
truncated resolvent series on the same moments: exact and probing moments,
with and without Gutzwiller weights; FP64 <= 1e-10 relative to the largest
value, FP32 <= 1e-4."""
import numpy as np
import pytest

from oracle import bdg, ldos, rmft
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


def _setup(K, nx, ny, M):
    kpm, ctx = K
    N = nx * ny
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, p, 0.3, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    return model, p, fields, ab


OMEGA = np.array([-0.8, -0.3, -0.05, 0.0, 0.02, 0.2, 0.7])


@pytest.mark.parametrize("prec,weighted,probe", [("fp64", False, 0), ("fp64", True, 0), ("fp32", True, 0),
                                                  ("fp64", True, 2)])
def test_ldos_matches_oracle(K, prec, weighted, probe):
    kpm, ctx = K
    nx, ny, M = 8, 6, 384
    N = nx * ny
    model, p, fields, ab = _setup(K, nx, ny, M)
    P = kpm.KPM_FP64 if prec == "fp64" else kpm.KPM_FP32
    out = torch.empty(2 * len(OMEGA) * N, dtype=torch.float64, device="cuda")
    kpm.kpm_ldos(ctx, model, kpm.make_opts(M, P, probe_p=probe, probe_seed=3), fields, ab,
                 p if weighted else None, OMEGA, out, gamma_alpha=0.25, gamma0=0.02)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(2, len(OMEGA), N)
    o = rmft.Model(nx, ny)
    a, b = ab.cpu().numpy()
    h = bdg.dense(o, fields.cpu().numpy())
    mu = ldos.moments_probing(h, a, b, M, nx, ny, probe, 3) if probe else ldos.moments(h, a, b, M)
    wgt = ldos.gutzwiller_weights(p.cpu().numpy(), N) if weighted else None
    ref = ldos.ldos_from_moments(mu, a, b, OMEGA, 0.25, 0.02, wgt)
    tol = (1e-10 if prec == "fp64" else 1e-4) * np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) < tol


def test_ldos_converges_to_the_lorentzians(K):
    kpm, ctx = K
    nx, ny, M = 8, 6, 4096
    N = nx * ny
    model, p, fields, ab = _setup(K, nx, ny, M)
    out = torch.empty(2 * len(OMEGA) * N, dtype=torch.float64, device="cuda")
    kpm.kpm_ldos(ctx, model, kpm.make_opts(M, kpm.KPM_FP64), fields, ab, None, OMEGA, out, 0.25, 0.05)
    torch.cuda.synchronize()
    ex = ldos.ldos_exact(bdg.dense(rmft.Model(nx, ny), fields.cpu().numpy()), OMEGA, 0.25, 0.05)
    assert np.max(np.abs(out.cpu().numpy().reshape(2, len(OMEGA), N) - ex)) < 1e-8 * np.max(ex)
