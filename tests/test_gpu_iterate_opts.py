"""Options of rmft_iterate on the GPU, through the C ABI:

- strict: KPM_ENOTCONV when n_iter iterations end without meeting tol, with
  the parameters as after the last iteration;
- sync_every: k iterations queued per host read give the same parameters,
  statistics and iteration count as one read per iteration, also when the
  loop converges inside a group (the device freezes the converged state);
- anderson: the Anderson-mixed trajectory (reading R4) follows the oracle's
  for 14 iterations (FP64, 1e-10);
- rmft_prepare / kpm_observables / rmft_update in sequence equal one
  rmft_iterate iteration bit for bit;
- kpm_measure_peaks reports positive FP64 and FP32 FMA rates.
"""
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


def _setup(K, nx, ny, M, delta=0.15, seed=3):
    kpm, ctx = K
    N = nx * ny
    w = inputs.Workload(nx, ny, delta, inputs.two_vortex(nx, ny), M, seed=seed)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    return w, model, phi, inputs.vortex_seed(w)


def test_strict_reports_not_converged(K):
    kpm, ctx = K
    w, model, phi, p0 = _setup(K, 8, 6, 32)
    p = torch.tensor(p0, device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, stats = kpm.rmft_iterate(ctx, model, kpm.make_opts(32, 0), kpm.make_rmft_opts(w.n_target, tol=1e-14,
                                                                                        strict=True),
                                 phi, p, mu, 2, check=False)
    assert st == kpm.KPM_ENOTCONV and stats.iterations == 2 and not stats.converged
    q = torch.tensor(p0, device="cuda")
    mq = torch.zeros(1, dtype=torch.float64, device="cuda")
    st2, _ = kpm.rmft_iterate(ctx, model, kpm.make_opts(32, 0), kpm.make_rmft_opts(w.n_target, tol=1e-14),
                              phi, q, mq, 2, check=False)
    assert st2 == kpm.KPM_OK and torch.equal(p, q)


@pytest.mark.parametrize("tol", [0.0, 0.03])
def test_sync_every_matches_one_read_per_iteration(K, tol):
    kpm, ctx = K
    w, model, phi, p0 = _setup(K, 12, 8, 64)
    opts = kpm.make_opts(64, kpm.KPM_FP32)
    res = []
    for k in (1, 7):
        p = torch.tensor(p0, device="cuda")
        mu = torch.zeros(1, dtype=torch.float64, device="cuda")
        _, st = kpm.rmft_iterate(ctx, model, opts, kpm.make_rmft_opts(w.n_target, tol=tol, sync_every=k), phi, p,
                                 mu, 40)
        res.append((p.cpu().numpy(), float(mu.item()), st))
    (pa, ma, sa), (pb, mb, sb) = res
    assert np.array_equal(pa, pb) and ma == mb
    for f in ("residual", "density_error", "mu", "omega", "a", "b", "iterations", "converged"):
        assert getattr(sa, f) == getattr(sb, f), f
    if tol > 0.0:
        assert sa.converged and sa.iterations < 40   # stopped inside a group of 7


def test_anderson_trajectory_matches_oracle(K):
    kpm, ctx = K
    w, model, phi, p0 = _setup(K, 10, 8, 64)
    p = torch.tensor(p0, device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    ro = kpm.make_rmft_opts(w.n_target, tol=0.0, anderson=4)
    traj = []
    # one call (the history lives for the duration of a call): 14 iterations,
    # read back one at a time through sync_every = 1 and the per-call stats
    _, st = kpm.rmft_iterate(ctx, model, kpm.make_opts(w.M, kpm.KPM_FP64), ro, phi, p, mu, 14)
    om = rmft.Model(w.nx, w.ny)
    x, m_eff = p0.copy(), 0.0
    mix = rmft.Anderson(4)
    for it in range(14):
        f, mu_phys = rmft.shifted_fields(om, x, m_eff)
        a, b = bdg.gershgorin(om, f)
        F1, omega = okpm.f_spectral(bdg.dense(om, f), a, b, w.M)
        x, m_eff, r, e = rmft.update_anderson(x, okpm.observables(om, F1), w.n_target, m_eff, mix)
    assert st.iterations == 14
    assert st.residual == pytest.approx(r, abs=1e-10)
    assert st.density_error == pytest.approx(e, abs=1e-10)
    assert np.max(np.abs(p.cpu().numpy() - x)) < 1e-10
    assert float(mu.item()) == pytest.approx(m_eff, abs=1e-10)


def test_split_iteration_equals_rmft_iterate(K):
    kpm, ctx = K
    w, model, phi, p0 = _setup(K, 9, 7, 48)
    N = w.n_sites
    opts = kpm.make_opts(48, kpm.KPM_FP32)
    ro = kpm.make_rmft_opts(w.n_target, tol=0.0)
    pa = torch.tensor(p0, device="cuda")
    ma = torch.zeros(1, dtype=torch.float64, device="cuda")
    kpm.rmft_iterate(ctx, model, opts, ro, phi, pa, ma, 2)
    pb = torch.tensor(p0, device="cuda")
    mb = torch.zeros(1, dtype=torch.float64, device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    muo = torch.empty(1, dtype=torch.float64, device="cuda")
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    stats = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        kpm.rmft_prepare(ctx, model, opts, phi, pb, mb, fields, ab, muo)
        kpm.kpm_observables(ctx, model, opts, fields, ab, obs)
        kpm.rmft_update(ctx, model, ro, pb, obs, mb, stats)
    torch.cuda.synchronize()
    assert torch.equal(pa, pb) and torch.equal(ma, mb)


def test_measured_peaks(K):
    kpm, ctx = K
    fp64, fp32, f32x2, mhz = kpm.kpm_measure_peaks(ctx)
    assert 0.1 < fp64 < 100.0
    assert fp32 > 5.0 * fp64 and f32x2 > 0.5 * fp32
    assert 500.0 < mhz < 3000.0
