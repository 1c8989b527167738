"""Batched self-consistency (rmft_iterate_batched) against per-cell iterations.

Cells of uneven shape, doping and vortex placement; the batched graph must
reproduce rmft_iterate cell by cell (same arithmetic, so to rounding), in
FP32 and FP64, and the first batched iterations of a cell must follow the
oracle's trajectory.
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
    return kpm


SHAPES = [(8, 6, 0.10), (10, 4, 0.2), (8, 6, 0.15), (6, 6, 0.25), (12, 6, 0.05), (10, 4, 0.3)]


def _cell(kpm, ctx, nx, ny, dop, seed):
    w = inputs.Workload(nx, ny, dop, inputs.two_vortex(nx, ny), 64, seed=seed)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * nx * ny, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    return w, model, phi, torch.tensor(inputs.vortex_seed(w), device="cuda")


@pytest.mark.parametrize("prec", [1, 0])
def test_batched_equals_per_cell(K, prec):
    kpm = K
    M = 64
    ctx_b = kpm.kpm_create(0)
    opts = kpm.make_opts(M, prec)
    cells = [_cell(kpm, ctx_b, nx, ny, d, k) for k, (nx, ny, d) in enumerate(SHAPES)]
    models = [c[1] for c in cells]
    phis = [c[2] for c in cells]
    params = [c[3].clone() for c in cells]
    ropts = [kpm.make_rmft_opts(c[0].n_target, tol=0.0) for c in cells]
    mu = torch.zeros(len(cells), dtype=torch.float64, device="cuda")
    _, stats = kpm.rmft_iterate_batched(ctx_b, models, opts, ropts, phis, params, mu, 3)
    torch.cuda.synchronize()
    tol = 1e-12
    for k, c in enumerate(cells):
        ctx = kpm.kpm_create(0)
        p = c[3].clone()
        m = torch.zeros(1, dtype=torch.float64, device="cuda")
        _, st = kpm.rmft_iterate(ctx, c[1], opts, ropts[k], c[2], p, m, 3)
        torch.cuda.synchronize()
        assert float((p - params[k]).abs().max()) < tol
        assert float(m.item()) == pytest.approx(float(mu[k].item()), abs=tol)
        assert stats[k].residual == pytest.approx(st.residual, abs=tol)
        assert stats[k].iterations == 3
        kpm.kpm_destroy(ctx)
    kpm.kpm_destroy(ctx_b)


def test_batched_cell_follows_oracle(K):
    kpm = K
    M = 48
    ctx = kpm.kpm_create(0)
    opts = kpm.make_opts(M, kpm.KPM_FP64)
    cells = [_cell(kpm, ctx, nx, ny, d, k) for k, (nx, ny, d) in enumerate(SHAPES[:4])]
    params = [c[3].clone() for c in cells]
    ropts = [kpm.make_rmft_opts(c[0].n_target, tol=0.0) for c in cells]
    mu = torch.zeros(len(cells), dtype=torch.float64, device="cuda")
    kpm.rmft_iterate_batched(ctx, [c[1] for c in cells], opts, ropts, [c[2] for c in cells], params, mu, 2)
    torch.cuda.synchronize()
    k = 1
    w = cells[k][0]
    om = rmft.Model(w.nx, w.ny)
    p, mu_eff = inputs.vortex_seed(w), 0.0
    for _ in range(2):
        f, _ = rmft.shifted_fields(om, p, mu_eff)
        a, b = bdg.gershgorin(om, f)
        F1, _ = okpm.f_spectral(bdg.dense(om, f), a, b, M)
        p, mu_eff, _, _ = rmft.update(p, okpm.observables(om, F1), w.n_target, mu_eff)
    assert np.max(np.abs(params[k].cpu().numpy() - p)) < 1e-10
    assert float(mu[k].item()) == pytest.approx(mu_eff, abs=1e-10)
    kpm.kpm_destroy(ctx)


def test_batched_cfg3_shapes_follow_oracle(K):
    """One cell of each shape of the 32-cell mix (24x12, 32x16, 48x24, 64x32;
    doping and seeds as drawn by cfg3_cells), FP32 at M = 1024 as benchmarked,
    one batched iteration: every site's updated n, chi, F, the residual and
    the density error against the oracle's shifted_fields -> f_spectral ->
    update chain (FP32 tolerance 2e-5)."""
    kpm = K
    cells = inputs.cfg3_cells(seed=0, count=32)
    pick = {}
    for w in cells:
        pick.setdefault((w.nx, w.ny), w)
    assert sorted(pick) == [(24, 12), (32, 16), (48, 24), (64, 32)]
    ws = [pick[s] for s in sorted(pick)]
    ctx = kpm.kpm_create(0)
    models, phis, params = [], [], []
    for w in ws:
        m = kpm.make_model(w.nx, w.ny)
        phi = torch.empty(4 * w.n_sites, dtype=torch.float64, device="cuda")
        kpm.kpm_peierls_phases(ctx, m, phi)
        models.append(m)
        phis.append(phi)
        params.append(torch.tensor(inputs.vortex_seed(w), device="cuda"))
    ropts = [kpm.make_rmft_opts(w.n_target, tol=0.0) for w in ws]
    mu = torch.zeros(len(ws), dtype=torch.float64, device="cuda")
    _, stats = kpm.rmft_iterate_batched(ctx, models, kpm.make_opts(1024, kpm.KPM_FP32), ropts, phis, params, mu, 1)
    torch.cuda.synchronize()
    for k, w in enumerate(ws):
        om = rmft.Model(w.nx, w.ny)
        p0 = inputs.vortex_seed(w)
        f, mu_phys = rmft.shifted_fields(om, p0, 0.0)
        a, b = bdg.gershgorin(om, f)
        F1, omega = okpm.f_spectral(bdg.dense(om, f), a, b, w.M)
        p1, mu1, r, e = rmft.update(p0, okpm.observables(om, F1), w.n_target, 0.0)
        got = params[k].cpu().numpy()
        assert np.max(np.abs(got - p1)) < 2e-5, (w.nx, w.ny)
        assert stats[k].residual == pytest.approx(r, abs=2e-5)
        assert stats[k].density_error == pytest.approx(e, abs=2e-5)
        assert stats[k].omega == pytest.approx(omega, rel=1e-5)
        assert float(mu[k].item()) == pytest.approx(mu1, abs=1e-5)
    kpm.kpm_destroy(ctx)
