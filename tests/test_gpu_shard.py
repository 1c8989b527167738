"""Site-range passes and the sharded driver on one GPU (the multi-GPU
partition of paper_2212_05685_gb300/shard.py, with every rank's range run in
turn on this device).

- kpm_observables over a partition of the sites: the obs sum to the full pass
  bit for bit (FP64 and FP32), the grand potentials to rounding, and the
  sites outside a range read zero;
- kpm_backward over the same partition: the gradients sum to the full
  gradient to rounding;
- the sharded loop with one rank (rmft_prepare, kpm_observables, rmft_update)
  equals rmft_iterate bit for bit;
- the site-range sums also match the oracle on sampled sites.
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


def _cell(K, nx, ny, M, seed=3):
    kpm, ctx = K
    N = nx * ny
    w = inputs.Workload(nx, ny, 0.15, inputs.two_vortex(nx, ny), M, seed=seed)
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p = inputs.vortex_seed(w)
    params = torch.tensor(p, device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.1, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    return w, model, phi, p, fields, ab


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("parts", [2, 3, 5])
def test_site_ranges_sum_to_full_pass(K, prec, parts):
    kpm, ctx = K
    from paper_2212_05685_gb300.shard import site_partition
    nx, ny, M = 20, 12, 96
    N = nx * ny
    w, model, _, _, fields, ab = _cell(K, nx, ny, M)
    full = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    om_full = torch.empty(1, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, kpm.make_opts(M, prec, block_width=100), fields, ab, full, om_full)
    acc = torch.zeros_like(full)
    om = 0.0
    for r in range(parts):
        b, e = site_partition(N, parts, r)
        part = torch.full_like(full, float("nan"))
        op = torch.empty(1, dtype=torch.float64, device="cuda")
        kpm.kpm_observables(ctx, model, kpm.make_opts(M, prec, block_width=100, site_begin=b, site_end=e),
                            fields, ab, part, op)
        n, chi, F = rmft.split(part.cpu().numpy(), N)
        outside = np.ones(N, dtype=bool)
        outside[b:e] = False
        assert not n[:, outside].any() and not chi[:, :, outside].any() and not F[:, outside].any()
        acc += part
        om += float(op.item())
    assert torch.equal(acc, full)
    assert om == pytest.approx(float(om_full.item()), rel=1e-12)


def test_site_range_matches_oracle(K):
    kpm, ctx = K
    nx, ny, M = 10, 8, 64
    N = nx * ny
    w, model, _, p, fields, ab = _cell(K, nx, ny, M, seed=5)
    out = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, kpm.make_opts(M, kpm.KPM_FP64, site_begin=17, site_end=41), fields, ab, out)
    om = rmft.Model(nx, ny)
    f = rmft.fields(om, p, 0.1)
    a, b = bdg.gershgorin(om, f)
    F1, _ = okpm.f_spectral(bdg.dense(om, f), a, b, M)
    ref = okpm.observables(om, F1)
    gn, gc, gF = rmft.split(out.cpu().numpy(), N)
    rn, rc, rF = rmft.split(ref, N)
    s = slice(17, 41)
    assert np.max(np.abs(gn[:, s] - rn[:, s])) < 1e-10
    assert np.max(np.abs(gc[:, :, s] - rc[:, :, s])) < 1e-10
    assert np.max(np.abs(gF[:, s] - rF[:, s])) < 1e-10


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-9)])
def test_backward_ranges_sum_to_full_gradient(K, prec, tol):
    kpm, ctx = K
    from paper_2212_05685_gb300.shard import site_partition
    nx, ny, M = 12, 8, 48
    N = nx * ny
    w, model, _, _, fields, ab = _cell(K, nx, ny, M, seed=6)
    g = torch.tensor(np.random.default_rng(2).uniform(-1, 1, size=26 * N), device="cuda")
    full = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_backward(ctx, model, kpm.make_opts(M, prec), fields, ab, g, 0.3, full, ckpt_every=8)
    acc = torch.zeros_like(full)
    for r in range(3):
        b, e = site_partition(N, 3, r)
        part = torch.empty_like(full)
        kpm.kpm_backward(ctx, model, kpm.make_opts(M, prec, site_begin=b, site_end=e), fields, ab, g, 0.3, part,
                         ckpt_every=8)
        acc += part
    scale = float(full.abs().max())
    assert float((acc - full).abs().max()) <= tol * scale


@pytest.mark.parametrize("prec", [0, 1])
def test_sharded_loop_one_rank_equals_rmft_iterate(K, prec):
    kpm, ctx = K
    from paper_2212_05685_gb300 import shard
    nx, ny, M = 16, 12, 64
    N = nx * ny
    w, model, phi, p, _, _ = _cell(K, nx, ny, M, seed=7)
    opts = kpm.make_opts(M, prec)
    ro = kpm.make_rmft_opts(w.n_target, tol=0.0)
    pa = torch.tensor(p, device="cuda")
    ma = torch.zeros(1, dtype=torch.float64, device="cuda")
    _, st = kpm.rmft_iterate(ctx, model, opts, ro, phi, pa, ma, 3)
    pb = torch.tensor(p, device="cuda")
    mb = torch.zeros(1, dtype=torch.float64, device="cuda")
    be = shard.DeviceBackend(ctx, model, opts, ro, phi, pb, mb)
    last, done = shard.rmft_iterate_sharded(be, shard.Comm(), 3)
    assert done == 3
    assert torch.equal(pa, pb) and torch.equal(ma, mb)
    assert last.residual == st.residual and last.density_error == st.density_error
    assert last.mu == st.mu and last.omega == st.omega


def test_site_range_refusals(K):
    kpm, ctx = K
    nx, ny, M = 6, 4, 16
    N = nx * ny
    w, model, phi, p, fields, ab = _cell(K, nx, ny, M)
    out = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    for sb, se, extra in ((5, 5, {}), (-1, 3, {}), (0, N + 1, {}), (2, 9, {"probe_p": 2}),
                          (2, 9, {"flags": kpm.KPM_FLAG_PH_HALF})):
        with pytest.raises(kpm.KPMError) as e:
            kpm.kpm_observables(ctx, model, kpm.make_opts(M, 1, site_begin=sb, site_end=se, **extra), fields, ab, out)
        assert e.value.status == kpm.KPM_EINVAL
    pa = torch.tensor(p, device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, _ = kpm.rmft_iterate(ctx, model, kpm.make_opts(M, 1, site_begin=0, site_end=5),
                             kpm.make_rmft_opts(w.n_target), phi, pa, mu, 1, check=False)
    assert st == kpm.KPM_EINVAL
