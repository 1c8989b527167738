"""Probing estimate on the GPU (App. B, reading P2) against the oracle's
probing estimate: FP64 <= 1e-10, FP32 <= 2e-5 on every observable; singleton
colours reproduce the exact unit-vector pass; an RMFT iteration with probing
follows the oracle's; invalid colourings are refused."""
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


def _setup(K, nx, ny, seed=0):
    kpm, ctx = K
    N = nx * ny
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64, seed=seed)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p = inputs.random_params(nx, ny, seed + 1)
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, torch.tensor(p, device="cuda"), 0.3, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    return model, phi, p, fields, ab


def _gpu(K, model, fields, ab, opts):
    kpm, ctx = K
    N = model.nx * model.ny
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    om = torch.empty(1, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, opts, fields, ab, obs, om)
    torch.cuda.synchronize()
    return obs.cpu().numpy(), float(om.item())


@pytest.mark.parametrize("nx,ny,p,M,bw,seed", [(12, 12, 3, 64, 0, 5), (12, 8, 2, 48, 0, 1), (18, 12, 6, 40, 24, 7),
                                               (16, 16, 4, 33, 0, 0)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_probing_matches_oracle(K, nx, ny, p, M, bw, seed, prec):
    kpm, _ = K
    model, phi, params, fields, ab = _setup(K, nx, ny, seed)
    P = kpm.KPM_FP64 if prec == "fp64" else kpm.KPM_FP32
    got, om = _gpu(K, model, fields, ab, kpm.make_opts(M, P, bw, probe_p=p, probe_seed=seed))
    o = rmft.Model(nx, ny)
    a, b = ab.cpu().numpy()
    ref, omega = probing.observables_probing(o, bdg.dense(o, fields.cpu().numpy()), a, b, M, p, seed)
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.max(np.abs(got - ref)) < tol
    assert om == pytest.approx(omega, rel=1e-10 if prec == "fp64" else 1e-5)


def test_singleton_colours_equal_the_exact_pass(K):
    kpm, _ = K
    nx = ny = 6
    model, phi, params, fields, ab = _setup(K, nx, ny, 2)
    exact, om = _gpu(K, model, fields, ab, kpm.make_opts(64, kpm.KPM_FP64))
    est, om2 = _gpu(K, model, fields, ab, kpm.make_opts(64, kpm.KPM_FP64, probe_p=6, probe_seed=9))
    assert np.max(np.abs(est - exact)) < 1e-12
    assert om2 == pytest.approx(om, rel=1e-12)


def test_probing_iteration_follows_oracle(K):
    kpm, ctx = K
    nx, ny, M, pr, seed = 12, 12, 64, 3, 4
    N = nx * ny
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p0 = inputs.vortex_seed(w)
    pd = torch.tensor(p0, device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    opts = kpm.make_opts(M, kpm.KPM_FP64, probe_p=pr, probe_seed=seed)
    ro = kpm.make_rmft_opts(w.n_target, tol=0.0)
    om_ = rmft.Model(nx, ny)
    pc, mu_eff = p0.copy(), 0.0
    for it in range(3):
        _, st = kpm.rmft_iterate(ctx, model, opts, ro, phi, pd, mu, 1)
        f, mu_phys = rmft.shifted_fields(om_, pc, mu_eff)
        a, b = bdg.gershgorin(om_, f)
        obs, omega = probing.observables_probing(om_, bdg.dense(om_, f), a, b, M, pr, seed)
        pc, mu_eff, r, e = rmft.update(pc, obs, w.n_target, mu_eff)
        assert st.residual == pytest.approx(r, abs=1e-10)
        assert st.omega == pytest.approx(omega, rel=1e-11)
    assert np.max(np.abs(pd.cpu().numpy() - pc)) < 1e-10


def test_invalid_colourings_are_refused(K):
    kpm, _ = K
    model, phi, params, fields, ab = _setup(K, 12, 8, 0)
    for bad in (dict(probe_p=1), dict(probe_p=5), dict(probe_p=3),  # 3 does not divide 8
                dict(probe_p=2, flags=kpm.KPM_FLAG_PH_HALF)):
        with pytest.raises(kpm.KPMError):
            _gpu(K, model, fields, ab, kpm.make_opts(32, kpm.KPM_FP64, **bad))


def test_full_size_probing_sampled_colours(K):
    """100 x 100 two-vortex cell with the PDW seed, M = 2048, FP32, p = 10
    (R = 200) as benchmarked: every site of two colour classes against the
    oracle's recursion on those probing vectors."""
    kpm, ctx = K
    w = inputs.CFG2
    nx, ny, N = w.nx, w.ny, w.n_sites
    p = inputs.vortex_seed(w)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, torch.tensor(p, device="cuda"), 0.0, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    got, _ = _gpu(K, model, fields, ab, kpm.make_opts(w.M, kpm.KPM_FP32, probe_p=10, probe_seed=1))
    orm = rmft.Model(nx, ny)
    f = rmft.fields(orm, p, 0.0)
    a, b = bdg.gershgorin(orm, f)
    assert ab.cpu().numpy() == pytest.approx([a, b], rel=1e-13)
    colours = [0, 1, 146, 147]  # both Nambu rows of the sites (x, y) = (0, 0) and (3, 7) mod 10
    J, F = probing.columns_probing_naive(bdg.csr(orm, f), a, b, w.M, nx, ny, 10, 1, colours)
    full = np.zeros((2 * N, 2 * N), dtype=np.complex128, order="F")
    full[:, J] = F
    ref = okpm.observables(orm, full)
    sites = np.unique(J // 2)
    assert len(sites) == 200
    gn, gc, gF = rmft.split(got, N)
    rn, rc, rF = rmft.split(ref, N)
    assert np.max(np.abs(gn[:, sites] - rn[:, sites])) < 2e-5
    assert np.max(np.abs(gc[:, :, sites] - rc[:, :, sites])) < 2e-5
    assert np.max(np.abs(gF[:, sites] - rF[:, sites])) < 2e-5
