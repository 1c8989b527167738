"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances: FP64 recursion <= 1e-10 absolute on every order parameter; FP32
recursion (FP64 moment sums) <= 2e-5 absolute.  Sizes span several CTA tiles
and column chunks, with ragged slabs (D not a multiple of the chunk or of the
slab width) and the degenerate orders M = 1, 2, 3.
"""
import numpy as np
import pytest

from oracle import bdg, kpm as okpm, kspace, rmft
from paper_2212_05685_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 2e-5


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_05685_gb300 import build, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    yield kpm, ctx
    kpm.kpm_destroy(ctx)


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def gpu_fields(K, nx, ny, p, mu, flux=1, gutz=True):
    kpm, ctx = K
    N = nx * ny
    model = kpm.make_model(nx, ny, flux=flux, gutzwiller=gutz)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    w = torch.empty(1, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, dev(p), mu, fields, w)
    return model, phi, fields, w


def gpu_pass(K, model, fields, M, prec, block_width=0, margin=0.01, cols=0):
    kpm, ctx = K
    N = model.nx * model.ny
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, margin, ab)
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    om = torch.empty(1, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, kpm.make_opts(M, prec, block_width, cols), fields, ab, obs, om)
    torch.cuda.synchronize()
    return obs.cpu().numpy(), float(om.item()), ab.cpu().numpy()


def oracle_pass(nx, ny, p, mu, M, flux=1, gutz=True):
    om = rmft.Model(nx, ny, flux=flux, gutzwiller=gutz)
    f = rmft.fields(om, p, mu)
    a, b = bdg.gershgorin(om, f)
    F1, omega = okpm.f_spectral(bdg.dense(om, f), a, b, M)
    return okpm.observables(om, F1), omega, (a, b), f


@pytest.mark.parametrize("nx,ny,flux", [(16, 16, 1), (48, 24, 1), (5, 7, 2), (3, 2, 1)])
def test_peierls_phases(K, nx, ny, flux):
    kpm, ctx = K
    N = nx * ny
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, kpm.make_model(nx, ny, flux=flux), phi)
    from oracle.lattice import peierls_phases
    assert np.max(np.abs(phi.cpu().numpy() - peierls_phases(nx, ny, flux).reshape(-1))) < 1e-13


@pytest.mark.parametrize("gutz,split,seed", [(True, 0.0, 1), (True, 0.03, 2), (False, 0.02, 3)])
def test_fields_and_W(K, gutz, split, seed):
    nx, ny = 7, 5
    p = inputs.random_params(nx, ny, seed, spin_split=split)
    model, phi, fields, w = gpu_fields(K, nx, ny, p, 0.37, gutz=gutz)
    om = rmft.Model(nx, ny, gutzwiller=gutz)
    ref = rmft.fields(om, p, 0.37)
    # FP64 on both sides, different summation order: relative 1e-13
    g = fields.cpu().numpy()
    assert np.max(np.abs(g - ref) / np.maximum(1.0, np.abs(ref))) < 1e-13
    assert float(w.item()) == pytest.approx(rmft.energy_W(om, p, 0.37), rel=1e-13, abs=1e-11)


def test_bounds(K):
    kpm, ctx = K
    nx, ny = 9, 6
    p = inputs.random_params(nx, ny, 4)
    model, phi, fields, _ = gpu_fields(K, nx, ny, p, 0.2)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    a, b = bdg.gershgorin(rmft.Model(nx, ny), rmft.fields(rmft.Model(nx, ny), p, 0.2))
    assert ab.cpu().numpy() == pytest.approx([a, b], rel=1e-13, abs=1e-14)


CASES = [
    # nx, ny, M, block_width (0 = whole D), seed kind
    (4, 4, 32, 0, "rand"),
    (5, 3, 40, 0, "rand"),      # D = 30: ragged against every column chunk
    (7, 5, 64, 7, "rand"),      # 10 slabs of 7 columns, the last one of 0 + ragged
    (16, 16, 256, 0, "vortex"),  # the 16 x 16 two-vortex cell at M = 256
    (16, 16, 256, 100, "vortex"),
    (12, 9, 97, 33, "vortex"),
]


def _params(nx, ny, kind, seed=7):
    if kind == "rand":
        return inputs.random_params(nx, ny, seed)
    return inputs.vortex_seed(inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64, seed=seed))


@pytest.mark.parametrize("nx,ny,M,bw,kind", CASES)
def test_observables_fp64(K, nx, ny, M, bw, kind):
    kpm, _ = K
    p = _params(nx, ny, kind)
    model, _, fields, _ = gpu_fields(K, nx, ny, p, 0.25)
    obs, om, ab = gpu_pass(K, model, fields, M, kpm.KPM_FP64, bw)
    ref, omega, (a, b), _ = oracle_pass(nx, ny, p, 0.25, M)
    assert ab == pytest.approx([a, b], rel=1e-13, abs=1e-14)
    assert np.max(np.abs(obs - ref)) < FP64_TOL
    assert om == pytest.approx(omega, rel=1e-11, abs=1e-10)


@pytest.mark.parametrize("nx,ny,M,bw,kind", CASES)
def test_observables_fp32(K, nx, ny, M, bw, kind):
    kpm, _ = K
    p = _params(nx, ny, kind)
    model, _, fields, _ = gpu_fields(K, nx, ny, p, 0.25)
    obs, om, _ = gpu_pass(K, model, fields, M, kpm.KPM_FP32, bw)
    ref, omega, _, _ = oracle_pass(nx, ny, p, 0.25, M)
    assert np.max(np.abs(obs - ref)) < FP32_TOL
    assert om == pytest.approx(omega, rel=1e-5)


@pytest.mark.parametrize("cols", [1, 2, 4, 8, 16])
def test_every_column_chunk_width(K, cols):
    kpm, _ = K
    nx, ny, M = 6, 5, 48
    p = _params(nx, ny, "rand", 9)
    model, _, fields, _ = gpu_fields(K, nx, ny, p, 0.1)
    ref, _, _, _ = oracle_pass(nx, ny, p, 0.1, M)
    for prec, tol in ((kpm.KPM_FP64, FP64_TOL), (kpm.KPM_FP32, FP32_TOL)):
        if prec == kpm.KPM_FP64 and cols > 8:
            continue
        obs, _, _ = gpu_pass(K, model, fields, M, prec, cols=cols)
        assert np.max(np.abs(obs - ref)) < tol


@pytest.mark.parametrize("M", [1, 2, 3])
def test_lowest_orders(K, M):
    kpm, _ = K
    nx, ny = 5, 4
    p = _params(nx, ny, "rand", 11)
    model, _, fields, _ = gpu_fields(K, nx, ny, p, 0.0)
    ref, omega, _, _ = oracle_pass(nx, ny, p, 0.0, M)
    obs, om, _ = gpu_pass(K, model, fields, M, kpm.KPM_FP64)
    assert np.max(np.abs(obs - ref)) < FP64_TOL
    assert om == pytest.approx(omega, rel=1e-12, abs=1e-12)


def test_rmft_trajectory_cfg0(K):
    """20 fixed-point iterations on the 16 x 16 two-vortex cell (M = 256)."""
    kpm, ctx = K
    w = inputs.CFG0
    nx, ny, N = w.nx, w.ny, w.n_sites
    p0 = inputs.vortex_seed(w)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = dev(p0)
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    ro = kpm.make_rmft_opts(w.n_target, tol=0.0)
    traj = []
    for it in range(20):
        _, st = kpm.rmft_iterate(ctx, model, kpm.make_opts(w.M, kpm.KPM_FP64), ro, phi, params, mu, 1)
        traj.append((st.residual, st.density_error, st.mu, st.omega))
    # oracle
    om = rmft.Model(nx, ny)
    p, mu_eff = p0.copy(), 0.0
    for it in range(20):
        f, mu_phys = rmft.shifted_fields(om, p, mu_eff)
        a, b = bdg.gershgorin(om, f)
        F1, omega = okpm.f_spectral(bdg.dense(om, f), a, b, w.M)
        p, mu_eff, r, e = rmft.update(p, okpm.observables(om, F1), w.n_target, mu_eff)
        g = traj[it]
        assert g[0] == pytest.approx(r, abs=1e-10)
        assert g[1] == pytest.approx(e, abs=1e-10)
        assert g[2] == pytest.approx(mu_phys, abs=1e-10)
        assert g[3] == pytest.approx(omega, rel=1e-11)
    assert np.max(np.abs(params.cpu().numpy() - p)) < FP64_TOL
    assert float(mu.item()) == pytest.approx(mu_eff, abs=1e-10)


def test_rmft_host_buffers_match_device(K):
    kpm, ctx = K
    nx, ny, M = 10, 8, 64
    w = inputs.Workload(nx, ny, 0.15, inputs.two_vortex(nx, ny), M)
    p0 = inputs.vortex_seed(w)
    N = nx * ny
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    ro = kpm.make_rmft_opts(w.n_target, tol=0.0)
    opts = kpm.make_opts(M, kpm.KPM_FP32)
    pd = dev(p0)
    md = torch.zeros(1, dtype=torch.float64, device="cuda")
    kpm.rmft_iterate(ctx, model, opts, ro, phi, pd, md, 3)
    ph = p0.copy()
    mh = np.zeros(1)
    kpm.rmft_iterate(ctx, model, opts, ro, phi.cpu().numpy(), ph, mh, 3)
    assert np.array_equal(pd.cpu().numpy(), ph)
    assert float(md.item()) == mh[0]


@pytest.mark.parametrize("prec,M,tol", [("fp32", 2048, FP32_TOL), ("fp64", 64, FP64_TOL)])
def test_full_size_uniform_against_momentum_space(K, prec, M, tol):
    """100 x 100 (D = 20000), zero field: every site against the k-space closed form."""
    kpm, _ = K
    nx = ny = 100
    p = inputs.uniform_dwave(nx, ny, 0.125, chi_nn=0.19, chi_nnn=0.01, pair=0.12)
    model, _, fields, _ = gpu_fields(K, nx, ny, p, 0.0, flux=0)
    obs, om, ab = gpu_pass(K, model, fields, M, kpm.KPM_FP32 if prec == "fp32" else kpm.KPM_FP64)
    f = rmft.fields(rmft.Model(nx, ny, flux=0), p, 0.0)
    a, b = bdg.gershgorin(rmft.Model(nx, ny, flux=0), f)
    ref, omega = kspace.kpm_uniform(nx, ny, kspace.site_fields(f, nx * ny), a, b, M)
    assert np.max(np.abs(obs - ref)) < tol
    assert om == pytest.approx(omega, rel=1e-5 if prec == "fp32" else 1e-11)


def test_full_size_vortex_sampled_columns(K):
    """100 x 100 two-vortex cell with the PDW seed, M = 2048, FP32 as benchmarked:
    112 sites (224 unit columns) against the oracle's recursion on their columns:
    both vortex cores with their neighbours, four corners of the cell, and
    sites drawn across the lattice (oracle columns on spawn-started processes)."""
    import os
    from oracle import pool
    kpm, _ = K
    w = inputs.CFG2
    nx, ny, N = w.nx, w.ny, w.n_sites
    p = inputs.vortex_seed(w)
    model, _, fields, _ = gpu_fields(K, nx, ny, p, 0.0)
    obs, om, ab = gpu_pass(K, model, fields, w.M, kpm.KPM_FP32)
    orm = rmft.Model(nx, ny)
    a, b = bdg.gershgorin(orm, rmft.fields(orm, p, 0.0))
    assert ab == pytest.approx([a, b], rel=1e-13)
    sites = pool.sample_sites(nx, ny, 108, w.vortices, seed=5)
    sites = np.unique(np.concatenate([sites, [0, nx - 1, N - nx, N - 1]]))
    assert len(sites) >= 100
    workers = max(1, min(16, len(os.sched_getaffinity(0))))
    cp = pool.ColumnPool(nx, ny, p, 0.0, w.M, workers)
    try:
        rn, rc, rF, _ = cp.site_observables(sites)
    finally:
        cp.close()
    gn, gc, gF = rmft.split(obs, N)
    assert np.max(np.abs(gn[:, sites] - rn)) < FP32_TOL
    assert np.max(np.abs(gc[:, :, sites] - rc)) < FP32_TOL
    assert np.max(np.abs(gF[:, sites] - rF)) < FP32_TOL


def test_invalid_arguments_are_refused(K):
    kpm, ctx = K
    lib = ctx.lib
    import ctypes
    m = kpm.make_model(4, 4)
    host = np.zeros(4 * 16)
    assert lib.kpm_peierls_phases(ctx.handle, ctypes.byref(m), host.ctypes.data_as(ctypes.c_void_p), None) == kpm.KPM_EINVAL
    bad = kpm.make_model(1, 4)
    d = torch.zeros(64, dtype=torch.float64, device="cuda")
    assert lib.kpm_peierls_phases(ctx.handle, ctypes.byref(bad), ctypes.c_void_p(d.data_ptr()), None) == kpm.KPM_EINVAL
    f = torch.zeros(26 * 16, dtype=torch.float64, device="cuda")
    ab = torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda")
    o = kpm.make_opts(0, kpm.KPM_FP64)
    st = lib.kpm_observables(ctx.handle, ctypes.byref(m), ctypes.byref(o), ctypes.c_void_p(f.data_ptr()),
                             ctypes.c_void_p(ab.data_ptr()), ctypes.c_void_p(f.data_ptr()), None, None)
    assert st == kpm.KPM_EINVAL
