"""Particle-hole half pass (KPM_FLAG_PH_HALF): only the columns (j, up) are
propagated; in the paramagnetic singlet sector the result equals the full
pass and the oracle (App. B, readings N1-N4).  Refusals outside the sector."""
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


def _fields(K, nx, ny, p, mu=0.0):
    kpm, ctx = K
    N = nx * ny
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, torch.tensor(p, device="cuda"), mu, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    return model, phi, fields, ab


def _pass(K, model, fields, ab, M, prec, flags):
    kpm, ctx = K
    N = model.nx * model.ny
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    om = torch.empty(1, dtype=torch.float64, device="cuda")
    st = kpm.kpm_observables(ctx, model, kpm.make_opts(M, prec, flags=flags), fields, ab, obs, om)
    torch.cuda.synchronize()
    return st, obs.cpu().numpy(), float(om.item())


@pytest.mark.parametrize("nx,ny,M", [(10, 8, 96), (13, 7, 65)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_half_pass_matches_oracle_and_full_pass(K, nx, ny, M, prec):
    kpm, _ = K
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M)
    model, phi, fields, ab = _fields(K, nx, ny, inputs.vortex_seed(w), 0.4)
    P = kpm.KPM_FP64 if prec == "fp64" else kpm.KPM_FP32
    _, half, om_h = _pass(K, model, fields, ab, M, P, kpm.KPM_FLAG_PH_HALF)
    _, full, om_f = _pass(K, model, fields, ab, M, P, 0)
    o = rmft.Model(nx, ny)
    a, b = ab.cpu().numpy()
    F1, omega = okpm.f_spectral(bdg.dense(o, fields.cpu().numpy()), a, b, M)
    ref = okpm.observables(o, F1)
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.max(np.abs(half - ref)) < tol
    assert np.max(np.abs(half - full)) < tol
    assert om_h == pytest.approx(omega, rel=1e-11 if prec == "fp64" else 1e-5)
    N = nx * ny
    assert np.array_equal(half[:N], half[N:2 * N])          # n_dn = n_up
    assert np.array_equal(half[2 * N:10 * N], half[10 * N:18 * N])  # chi_dn = chi_up
    F = half[18 * N:].reshape(4, N, 2)
    nn = rmft.Model(nx, ny).nn4
    for e in range(4):  # F_{j,j+e} = F_{j+e,j} exactly
        assert np.array_equal(F[e], F[(e + 2) % 4][nn[e]])


def test_half_iterations_stay_in_the_sector(K):
    """FP32, one iteration per call (each call re-checks the sector)."""
    kpm, ctx = K
    nx, ny, M = 24, 12, 128
    N = nx * ny
    w = inputs.Workload(nx, ny, 0.15, inputs.two_vortex(nx, ny), M, pdw=0.02)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p = torch.tensor(inputs.vortex_seed(w), device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    opts = kpm.make_opts(M, kpm.KPM_FP32, flags=kpm.KPM_FLAG_PH_HALF)
    for _ in range(6):
        kpm.rmft_iterate(ctx, model, opts, kpm.make_rmft_opts(w.n_target, tol=0.0), phi, p, mu, 1)
    q = p.cpu().numpy()
    assert np.array_equal(q[:N], q[N:2 * N])
    assert np.array_equal(q[2 * N:10 * N], q[10 * N:18 * N])


def test_half_iteration_follows_full_iteration(K):
    """Ten FP64 RMFT iterations of the 16 x 16 two-vortex cell: the half pass
    follows the full pass (and does half the recursion bytes)."""
    kpm, ctx = K
    w = inputs.CFG0
    N = w.n_sites
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    out = {}
    for flags in (0, kpm.KPM_FLAG_PH_HALF):
        p = torch.tensor(inputs.vortex_seed(w), device="cuda")
        mu = torch.zeros(1, dtype=torch.float64, device="cuda")
        st, stats = kpm.rmft_iterate(ctx, model, kpm.make_opts(w.M, kpm.KPM_FP64, flags=flags),
                                     kpm.make_rmft_opts(w.n_target, tol=0.0), phi, p, mu, 10)
        assert st == kpm.KPM_OK
        torch.cuda.synchronize()
        out[flags] = (p.cpu().numpy(), float(mu.item()), stats)
    (p0, m0, s0), (p1, m1, s1) = out[0], out[kpm.KPM_FLAG_PH_HALF]
    assert np.max(np.abs(p0 - p1)) < 1e-10
    assert m0 == pytest.approx(m1, abs=1e-10)
    assert s1.omega == pytest.approx(s0.omega, rel=1e-11)
    assert s1.recursion_bytes == pytest.approx(0.5 * s0.recursion_bytes, rel=1e-12)


def test_half_pass_refused_outside_the_sector(K):
    kpm, ctx = K
    nx, ny, M = 8, 6, 32
    N = nx * ny
    p = inputs.random_params(nx, ny, 2)  # spin-split: n_up != n_dn, chi_up != chi_dn
    model, phi, fields, ab = _fields(K, nx, ny, p, 0.2)
    half = kpm.make_opts(M, kpm.KPM_FP64, flags=kpm.KPM_FLAG_PH_HALF)
    with pytest.raises(kpm.KPMError, match="particle-hole"):
        _pass(K, model, fields, ab, M, kpm.KPM_FP64, kpm.KPM_FLAG_PH_HALF)
    pd = torch.tensor(p, device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, _ = kpm.rmft_iterate(ctx, model, half, kpm.make_rmft_opts(0.875), phi, pd, mu, 1, check=False)
    assert st == kpm.KPM_EINVAL
    assert torch.equal(pd, torch.tensor(p, device="cuda"))  # nothing was updated
    # symmetric fields but a shifted rescaling centre
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M)
    model, phi, fields, ab = _fields(K, nx, ny, inputs.vortex_seed(w), 0.2)
    ab2 = ab.clone()
    ab2[1] = 0.05
    with pytest.raises(kpm.KPMError, match="centre"):
        _pass(K, model, fields, ab2, M, kpm.KPM_FP64, kpm.KPM_FLAG_PH_HALF)
    # calls that do not take the flag
    g = torch.zeros(26 * N, dtype=torch.float64, device="cuda")
    gf = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    with pytest.raises(kpm.KPMError, match="kpm_backward"):
        kpm.kpm_backward(ctx, model, half, fields, ab, g, 0.0, gf)
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    assert kpm.kpm_observables_noalloc(model, half, fields, ab, obs) == kpm.KPM_EINVAL


def test_full_size_half_pass_sampled_sites(K):
    """100 x 100 two-vortex cell with the PDW seed, M = 2048, FP32, half pass
    as benchmarked: sites sampled across the lattice against the oracle's
    recursion on both of their columns (the oracle propagates the (j, dn)
    columns the GPU reconstructs from the particle-hole relation)."""
    kpm, _ = K
    w = inputs.CFG2
    nx, ny, N = w.nx, w.ny, w.n_sites
    p = inputs.vortex_seed(w)
    model, phi, fields, ab = _fields(K, nx, ny, p, 0.0)
    st, half, _ = _pass(K, model, fields, ab, w.M, kpm.KPM_FP32, kpm.KPM_FLAG_PH_HALF)
    assert st == kpm.KPM_OK
    orm = rmft.Model(nx, ny)
    f = rmft.fields(orm, p, 0.0)
    a, b = bdg.gershgorin(orm, f)
    assert ab.cpu().numpy() == pytest.approx([a, b], rel=1e-13, abs=1e-14)
    rng = np.random.default_rng(11)
    sites = np.concatenate([[0, nx - 1, N - 1, 25 + 50 * nx, 75 + 50 * nx], rng.choice(N, 3, replace=False)])
    cols = np.sort(np.concatenate([2 * sites, 2 * sites + 1]))
    Fc, _ = okpm.f_naive(bdg.csr(orm, f), a, b, w.M, cols=cols)
    full = np.zeros((2 * N, 2 * N), dtype=np.complex128, order="F")
    full[:, cols] = Fc
    ref = okpm.observables(orm, full)
    gn, gc, gF = rmft.split(half, N)
    rn, rc, rF = rmft.split(ref, N)
    assert np.max(np.abs(gn[:, sites] - rn[:, sites])) < 2e-5
    assert np.max(np.abs(gc[:, :, sites] - rc[:, :, sites])) < 2e-5
    assert np.max(np.abs(gF[:, sites] - rF[:, sites])) < 2e-5
