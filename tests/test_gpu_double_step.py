"""FP32 recursion two steps per launch (KPM_FLAG_DOUBLE_STEP) against one step
per launch (the default): the arithmetic is the same, so the results agree bit for bit; and
against the oracle (Eq. alpha, App. B).  Lattices with bands of 4..64 rows,
ragged column chunks and slabs, odd and even M."""
import numpy as np
import pytest

from oracle import bdg, kpm as okpm, rmft
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


def _iterate(K, nx, ny, M, bw, flags, n_iter=2):
    kpm, ctx = K
    N = nx * ny
    w = inputs.Workload(nx, ny, 0.15, inputs.two_vortex(nx, ny), M)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p = torch.tensor(inputs.vortex_seed(w), device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    _, st = kpm.rmft_iterate(ctx, model, kpm.make_opts(M, kpm.KPM_FP32, bw, flags=flags),
                             kpm.make_rmft_opts(w.n_target, tol=0.0), phi, p, mu, n_iter)
    torch.cuda.synchronize()
    return p.cpu().numpy(), float(mu.item()), st


@pytest.mark.parametrize("nx,ny,M,bw", [(24, 12, 64, 0), (20, 13, 33, 0), (48, 24, 65, 700), (64, 64, 8, 0),
                                        (100, 100, 7, 1000), (48, 24, 2, 0), (48, 24, 3, 0), (48, 24, 4, 0)])
def test_two_steps_per_launch_equal_one(K, nx, ny, M, bw):
    kpm, _ = K
    p2, mu2, st2 = _iterate(K, nx, ny, M, bw, kpm.KPM_FLAG_DOUBLE_STEP)
    p1, mu1, st1 = _iterate(K, nx, ny, M, bw, 0)
    assert np.array_equal(p1, p2)
    assert mu1 == mu2
    assert st1.omega == st2.omega
    D = 2 * nx * ny
    if M >= 4:
        # the double-step path streams fewer slab bytes with fewer launches
        assert st2.recursion_launches < st1.recursion_launches
        assert st2.recursion_bytes < st1.recursion_bytes


def test_double_step_pass_matches_oracle(K):
    kpm, ctx = K
    nx, ny, M = 20, 13, 96
    N = nx * ny
    p = inputs.random_params(nx, ny, 4)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, torch.tensor(p, device="cuda"), 0.3, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    om = torch.empty(1, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, kpm.make_opts(M, kpm.KPM_FP32, flags=kpm.KPM_FLAG_DOUBLE_STEP), fields, ab,
                        obs, om)
    torch.cuda.synchronize()
    o = rmft.Model(nx, ny)
    a, b = ab.cpu().numpy()
    F1, omega = okpm.f_spectral(bdg.dense(o, fields.cpu().numpy()), a, b, M)
    assert np.max(np.abs(obs.cpu().numpy() - okpm.observables(o, F1))) < 2e-5
    assert float(om.item()) == pytest.approx(omega, rel=1e-5)
