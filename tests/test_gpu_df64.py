"""Double-float recursion (KPM_DF64): vectors and 2h~ entries as unevaluated
sums hi + lo of two FP32 numbers, arithmetic on the FP32 pipes.  Held to the
FP64 bar against the oracle (1e-10 on every observable) on the cases of the
FP64 parity tests, every column chunk, the lowest orders, the half and
probing passes and T > 0, the full-size uniform cell against the k-space
closed form; an RMFT trajectory follows the FP64 one; the calls that do not
take it refuse it."""
import numpy as np
import pytest

from oracle import bdg, kpm as okpm, kspace, probing, rmft
from paper_2212_05685_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_05685_gb300 import build, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    yield kpm, ctx
    kpm.kpm_destroy(ctx)


def _fields(K, nx, ny, p, mu, flux=1):
    kpm, ctx = K
    N = nx * ny
    model = kpm.make_model(nx, ny, flux=flux)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, torch.tensor(np.asarray(p, dtype=np.float64), device="cuda"), mu, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    return model, phi, fields, ab


def _pass(K, model, fields, ab, opts):
    kpm, ctx = K
    N = model.nx * model.ny
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    om = torch.empty(1, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, opts, fields, ab, obs, om)
    torch.cuda.synchronize()
    return obs.cpu().numpy(), float(om.item())


def _params(nx, ny, kind, seed=7):
    if kind == "rand":
        return inputs.random_params(nx, ny, seed)
    return inputs.vortex_seed(inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64, seed=seed))


def _oracle(nx, ny, fields, ab, M, T=0.0):
    o = rmft.Model(nx, ny)
    a, b = ab.cpu().numpy()
    F1, omega = okpm.f_spectral(bdg.dense(o, fields.cpu().numpy()), a, b, M, T)
    return okpm.observables(o, F1), omega


@pytest.mark.parametrize("nx,ny,M,bw,kind", [(4, 4, 32, 0, "rand"), (5, 3, 40, 0, "rand"), (7, 5, 64, 7, "rand"),
                                             (16, 16, 256, 0, "vortex"), (16, 16, 256, 100, "vortex"),
                                             (12, 9, 97, 33, "vortex")])
def test_df64_matches_oracle(K, nx, ny, M, bw, kind):
    kpm, _ = K
    model, _, fields, ab = _fields(K, nx, ny, _params(nx, ny, kind), 0.25)
    got, om = _pass(K, model, fields, ab, kpm.make_opts(M, kpm.KPM_DF64, bw))
    ref, omega = _oracle(nx, ny, fields, ab, M)
    assert np.max(np.abs(got - ref)) < TOL
    assert om == pytest.approx(omega, rel=1e-11, abs=1e-10)


@pytest.mark.parametrize("cols", [1, 2, 4, 8])
def test_df64_every_column_chunk(K, cols):
    kpm, _ = K
    nx, ny, M = 6, 5, 48
    model, _, fields, ab = _fields(K, nx, ny, _params(nx, ny, "rand", 9), 0.1)
    got, _ = _pass(K, model, fields, ab, kpm.make_opts(M, kpm.KPM_DF64, cols_per_block=cols))
    ref, _ = _oracle(nx, ny, fields, ab, M)
    assert np.max(np.abs(got - ref)) < TOL


@pytest.mark.parametrize("M", [1, 2, 3])
def test_df64_lowest_orders(K, M):
    kpm, _ = K
    nx, ny = 5, 4
    model, _, fields, ab = _fields(K, nx, ny, _params(nx, ny, "rand", 11), 0.0)
    got, om = _pass(K, model, fields, ab, kpm.make_opts(M, kpm.KPM_DF64))
    ref, omega = _oracle(nx, ny, fields, ab, M)
    assert np.max(np.abs(got - ref)) < TOL
    assert om == pytest.approx(omega, rel=1e-12, abs=1e-12)


def test_df64_half_probing_and_temperature(K):
    kpm, _ = K
    nx, ny, M = 12, 12, 64
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M)
    model, _, fields, ab = _fields(K, nx, ny, inputs.vortex_seed(w), 0.0)
    ref, omega = _oracle(nx, ny, fields, ab, M)
    half, om_h = _pass(K, model, fields, ab, kpm.make_opts(M, kpm.KPM_DF64, flags=kpm.KPM_FLAG_PH_HALF))
    assert np.max(np.abs(half - ref)) < TOL
    assert om_h == pytest.approx(omega, rel=1e-11)
    o = rmft.Model(nx, ny)
    a, b = ab.cpu().numpy()
    est, om_p = _pass(K, model, fields, ab, kpm.make_opts(M, kpm.KPM_DF64, probe_p=3, probe_seed=4))
    pref, pom = probing.observables_probing(o, bdg.dense(o, fields.cpu().numpy()), a, b, M, 3, 4)
    assert np.max(np.abs(est - pref)) < TOL
    assert om_p == pytest.approx(pom, rel=1e-10)
    T = 0.1
    hot, om_t = _pass(K, model, fields, ab, kpm.make_opts(M, kpm.KPM_DF64, temperature=T))
    tref, tom = _oracle(nx, ny, fields, ab, M, T)
    assert np.max(np.abs(hot - tref)) < TOL
    assert om_t == pytest.approx(tom, rel=1e-10)


def test_df64_full_size_uniform_against_momentum_space(K):
    """100 x 100 (D = 20000), zero field, M = 64: every site against the k-space closed form."""
    kpm, _ = K
    nx = ny = 100
    p = inputs.uniform_dwave(nx, ny, 0.125, chi_nn=0.19, chi_nnn=0.01, pair=0.12)
    model, _, fields, ab = _fields(K, nx, ny, p, 0.0, flux=0)
    got, om = _pass(K, model, fields, ab, kpm.make_opts(64, kpm.KPM_DF64))
    f = rmft.fields(rmft.Model(nx, ny, flux=0), p, 0.0)
    a, b = bdg.gershgorin(rmft.Model(nx, ny, flux=0), f)
    ref, omega = kspace.kpm_uniform(nx, ny, kspace.site_fields(f, nx * ny), a, b, 64)
    assert np.max(np.abs(got - ref)) < TOL
    assert om == pytest.approx(omega, rel=1e-11)


def test_df64_against_fp64_at_m1024(K):
    """48 x 24 cell at its seeded order parameters, M = 1024: double-float
    and FP64 recursions agree to the FP64 bar."""
    kpm, _ = K
    w = inputs.CFG1
    model, _, fields, ab = _fields(K, w.nx, w.ny, inputs.vortex_seed(w), 1.7)
    d64, om64 = _pass(K, model, fields, ab, kpm.make_opts(w.M, kpm.KPM_FP64))
    ddf, omdf = _pass(K, model, fields, ab, kpm.make_opts(w.M, kpm.KPM_DF64))
    assert np.max(np.abs(ddf - d64)) < TOL
    assert omdf == pytest.approx(om64, rel=1e-12)


def test_df64_rmft_trajectory_follows_fp64(K):
    kpm, ctx = K
    w = inputs.CFG0
    N = w.n_sites
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    out = {}
    for prec in (kpm.KPM_FP64, kpm.KPM_DF64):
        p = torch.tensor(inputs.vortex_seed(w), device="cuda")
        mu = torch.zeros(1, dtype=torch.float64, device="cuda")
        st, stats = kpm.rmft_iterate(ctx, model, kpm.make_opts(w.M, prec), kpm.make_rmft_opts(w.n_target, tol=0.0),
                                     phi, p, mu, 5)
        assert st == kpm.KPM_OK
        torch.cuda.synchronize()
        out[prec] = (p.cpu().numpy(), float(mu.item()), stats.omega)
    (p0, m0, o0), (p1, m1, o1) = out[kpm.KPM_FP64], out[kpm.KPM_DF64]
    assert np.max(np.abs(p0 - p1)) < TOL
    assert m1 == pytest.approx(m0, abs=TOL)
    assert o1 == pytest.approx(o0, rel=1e-12)


def test_df64_refused_where_not_supported(K):
    kpm, ctx = K
    nx, ny, M = 6, 4, 16
    N = nx * ny
    model, phi, fields, ab = _fields(K, nx, ny, _params(nx, ny, "rand", 3), 0.1)
    o = kpm.make_opts(M, kpm.KPM_DF64)
    g = torch.zeros(26 * N, dtype=torch.float64, device="cuda")
    gf = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    with pytest.raises(kpm.KPMError, match="KPM_DF64"):
        kpm.kpm_backward(ctx, model, o, fields, ab, g, 0.0, gf)
    ld = torch.empty(2 * 3 * N, dtype=torch.float64, device="cuda")
    with pytest.raises(kpm.KPMError, match="KPM_DF64"):
        kpm.kpm_ldos(ctx, model, o, fields, ab, None, np.array([-0.1, 0.0, 0.1]), ld)
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    assert kpm.kpm_observables_noalloc(model, o, fields, ab, obs) == kpm.KPM_EINVAL
    p = torch.tensor(_params(nx, ny, "rand", 3), device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, _ = kpm.rmft_iterate_batched(ctx, [model], o, [kpm.make_rmft_opts(0.875)], [phi], [p], mu, 1, check=False)
    assert st == kpm.KPM_EINVAL
