"""GPU adjoint (kpm_backward) against the oracle and against finite differences.

FP64 backward within 1e-10 (relative to the largest gradient entry) of the
oracle's Daleckii-Krein gradient, on several lattices, slab widths and
checkpoint intervals; FP32 backward within 2e-5 relative; the grand
potential's gradient tends to the Hellmann-Feynman (ED density matrix)
closed form; directional finite differences of FP64 forward passes; the
64 x 64 cell at M = 1024 with checkpoints every 32 moments.
"""
import numpy as np
import pytest

from oracle import adjoint, bdg, kpm as okpm, rmft
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


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _prep(K, nx, ny, p, mu=0.2, flux=1):
    kpm, ctx = K
    N = nx * ny
    model = kpm.make_model(nx, ny, flux=flux)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = dev(p)
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, mu, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    return model, phi, params, fields, ab


def _gpu_grad(K, model, fields, ab, M, prec, g_obs, g_om, bw=0, ckpt=0, phi=None, params=None):
    kpm, ctx = K
    N = model.nx * model.ny
    out = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    gphi = torch.empty(4 * N, dtype=torch.float64, device="cuda") if phi is not None else None
    kpm.kpm_backward(ctx, model, kpm.make_opts(M, prec, bw), fields, ab, dev(g_obs), g_om, out,
                     phi, params, gphi, ckpt)
    torch.cuda.synchronize()
    return out.cpu().numpy(), (gphi.cpu().numpy() if gphi is not None else None)


@pytest.mark.parametrize("nx,ny,M,bw,ckpt", [(4, 4, 24, 0, 0), (5, 3, 40, 7, 3), (6, 5, 33, 0, 2),
                                              (7, 4, 64, 13, 8)])
def test_backward_fp64_matches_oracle(K, nx, ny, M, bw, ckpt):
    kpm, _ = K
    p = inputs.random_params(nx, ny, 3)
    model, phi, params, fields, ab = _prep(K, nx, ny, p)
    rng = np.random.default_rng(nx * ny)
    g_obs, g_om = rng.normal(size=26 * nx * ny), float(rng.normal())
    got, gphi = _gpu_grad(K, model, fields, ab, M, kpm.KPM_FP64, g_obs, g_om, bw, ckpt, phi, params)
    om = rmft.Model(nx, ny)
    f = fields.cpu().numpy()
    a, b = ab.cpu().numpy()
    ref = adjoint.vjp_dense(om, f, a, b, M, g_obs, g_om)
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(got - ref)) < 1e-10 * scale
    ref_phi = adjoint.phi_grad(om, p, got)
    assert np.max(np.abs(gphi - ref_phi)) < 1e-10 * max(1.0, np.max(np.abs(ref_phi)))


# lattices inside one 16 x 8 site tile, across ragged tiles in x and y, slabs
# whose column-pair count is not a multiple of the 8-pair stage
@pytest.mark.parametrize("nx,ny,M,bw,ckpt", [(12, 8, 128, 0, 12), (18, 10, 96, 40, 7), (33, 17, 64, 0, 0)])
def test_backward_fp32_matches_oracle(K, nx, ny, M, bw, ckpt):
    kpm, _ = K
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M)
    p = inputs.vortex_seed(w)
    model, phi, params, fields, ab = _prep(K, nx, ny, p)
    rng = np.random.default_rng(5)
    g_obs, g_om = rng.normal(size=26 * nx * ny), 0.7
    got, _ = _gpu_grad(K, model, fields, ab, M, kpm.KPM_FP32, g_obs, g_om, bw=bw, ckpt=ckpt)
    ref = adjoint.vjp_dense(rmft.Model(nx, ny), fields.cpu().numpy(), *ab.cpu().numpy(), M, g_obs, g_om)
    assert np.max(np.abs(got - ref)) < 2e-5 * max(1.0, np.max(np.abs(ref)))


def test_grand_potential_gradient_hellmann_feynman(K):
    """12 x 12 cell: dOmega_M/dfields against the ED density matrix (M -> inf)."""
    kpm, _ = K
    nx = ny = 12
    p = inputs.vortex_seed(inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64))
    model, phi, params, fields, ab = _prep(K, nx, ny, p, mu=0.0)
    om = rmft.Model(nx, ny)
    f = fields.cpu().numpy()
    F0, _ = okpm.f_ed(bdg.dense(om, f))
    hf = adjoint.field_grad_from_G(om, F0, 1.0)
    a, b = ab.cpu().numpy()
    zero = np.zeros(26 * nx * ny)
    errs = []
    for M in (128, 512, 2048):
        got, _ = _gpu_grad(K, model, fields, ab, M, kpm.KPM_FP64, zero, 1.0)
        # exact for the truncated series: the Daleckii-Krein gradient of Omega_M
        assert np.max(np.abs(got - adjoint.vjp_dense(om, f, a, b, M, zero, 1.0))) < 1e-10
        errs.append(np.max(np.abs(got - hf)))
    assert errs[0] > errs[1] > errs[2]


def test_directional_finite_differences(K):
    kpm, ctx = K
    nx, ny, M = 12, 12, 128
    p = inputs.vortex_seed(inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M))
    model, phi, params, fields, ab = _prep(K, nx, ny, p)
    N = nx * ny
    rng = np.random.default_rng(11)
    g_obs, g_om = rng.normal(size=26 * N), float(rng.normal())
    got, _ = _gpu_grad(K, model, fields, ab, M, kpm.KPM_FP64, g_obs, g_om)
    opts = kpm.make_opts(M, kpm.KPM_FP64)

    def L(f):
        obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        om = torch.empty(1, dtype=torch.float64, device="cuda")
        kpm.kpm_observables(ctx, model, opts, f, ab, obs, om)
        torch.cuda.synchronize()
        return float(np.dot(g_obs, obs.cpu().numpy()) + g_om * om.item())

    h = 1e-6
    for _ in range(3):
        v = rng.normal(size=26 * N)
        fd = (L(fields + h * dev(v)) - L(fields - h * dev(v))) / (2 * h)
        assert float(np.dot(got, v)) == pytest.approx(fd, rel=1e-6)


def test_density_loss_componentwise_finite_differences(K):
    """The adjoint workload's loss L = sum_i (n_i - n_target,i)^2 (seeded
    targets 1 - delta + 0.01 U(-1, 1)) on a 24 x 24 vortex cell: every one of
    16 seeded field components of the regenerating FP64 and FP32 gradients
    against central differences with h = 1e-6 of FP64 forward passes (a, b
    fixed); FP64 within 1e-7 of the largest entry, FP32 within 2e-5."""
    kpm, ctx = K
    nx, ny, M = 24, 24, 256
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M, seed=1)
    model, phi, params, fields, ab = _prep(K, nx, ny, inputs.vortex_seed(w), mu=0.0)
    N = nx * ny
    nt = dev(inputs.target_density(w, seed=1))
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")

    def grad(prec):
        kpm.kpm_observables(ctx, model, kpm.make_opts(M, prec, flags=kpm.KPM_FLAG_KEEP_TAIL), fields, ab, obs)
        n = obs[:N] + obs[N:2 * N]
        g = torch.zeros(26 * N, dtype=torch.float64, device="cuda")
        g[:N] = 2 * (n - nt)
        g[N:2 * N] = 2 * (n - nt)
        out = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        kpm.kpm_backward(ctx, model, kpm.make_opts(M, prec), fields, ab, g, 0.0, out, ckpt_every=kpm.KPM_REGENERATE)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    g64, g32 = grad(kpm.KPM_FP64), grad(kpm.KPM_FP32)
    o64 = kpm.make_opts(M, kpm.KPM_FP64)

    def L(f):
        kpm.kpm_observables(ctx, model, o64, f, ab, obs)
        n = obs[:N] + obs[N:2 * N]
        return float(((n - nt) ** 2).sum())

    h = 1e-6
    scale = float(np.abs(g64).max())
    assert scale > 0.0
    for k in np.random.default_rng(1).choice(26 * N, size=16, replace=False):
        f = fields.clone()
        f[int(k)] += h
        lp = L(f)
        f[int(k)] -= 2 * h
        fd = (lp - L(f)) / (2 * h)
        assert abs(g64[k] - fd) <= 1e-7 * scale, (int(k), g64[k], fd)
        assert abs(g32[k] - fd) <= 2e-5 * scale, (int(k), g32[k], fd)


def test_autograd_function(K):
    kpm, ctx = K
    from paper_2212_05685_gb300 import autograd
    nx, ny, M = 6, 4, 48
    model, phi, params, fields, ab = _prep(K, nx, ny, inputs.random_params(nx, ny, 8))
    f = fields.clone().requires_grad_(True)
    obs, om = autograd.observables(ctx, model, kpm.make_opts(M, kpm.KPM_FP64), f, ab)
    tgt = torch.linspace(0, 1, obs.numel(), dtype=torch.float64, device="cuda")
    loss = ((obs - tgt) ** 2).sum() + 0.3 * om.sum()
    loss.backward()
    g_obs = (2 * (obs - tgt)).detach().cpu().numpy()
    ref = adjoint.vjp_dense(rmft.Model(nx, ny), fields.cpu().numpy(), *ab.cpu().numpy(), M, g_obs, 0.3)
    assert np.max(np.abs(f.grad.cpu().numpy() - ref)) < 1e-10 * max(1.0, np.max(np.abs(ref)))


def test_adjoint_64x64_checkpoints_every_32(K):
    """The 64 x 64 adjoint workload: M = 1024, checkpoints every 32 moments,
    L = sum_i (n_i - n_target,i)^2, FP32 backward against FP64 forward
    directional differences."""
    kpm, ctx = K
    w = inputs.CFG4
    nx, ny, N, M = w.nx, w.ny, w.n_sites, w.M
    p = inputs.vortex_seed(w)
    model, phi, params, fields, ab = _prep(K, nx, ny, p, mu=0.0)
    nt = inputs.target_density(w, seed=1)
    o64 = kpm.make_opts(M, kpm.KPM_FP64)

    def forward(f, opts):
        obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        kpm.kpm_observables(ctx, model, opts, f, ab, obs)
        torch.cuda.synchronize()
        return obs.cpu().numpy()

    obs = forward(fields, kpm.make_opts(M, kpm.KPM_FP32))
    n = obs[:N] + obs[N:2 * N]
    g_obs = np.zeros(26 * N)
    g_obs[:N] = 2 * (n - nt)
    g_obs[N:2 * N] = 2 * (n - nt)
    got, _ = _gpu_grad(K, model, fields, ab, M, kpm.KPM_FP32, g_obs, 0.0, ckpt=32)

    def L(f):
        o = forward(f, o64)
        nn = o[:N] + o[N:2 * N]
        return float(np.sum((nn - nt) ** 2))

    rng = np.random.default_rng(1)
    h = 1e-5
    for _ in range(2):
        v = rng.normal(size=26 * N)
        fd = (L(fields + h * dev(v)) - L(fields - h * dev(v))) / (2 * h)
        assert float(np.dot(got, v)) == pytest.approx(fd, rel=2e-4)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_backward_is_deterministic(K, prec):
    """The stencil-entry sums use no atomics: two calls agree bit for bit."""
    kpm, ctx = K
    nx, ny, M = 12, 10, 96
    model, phi, params, fields, ab = _prep(K, nx, ny, inputs.random_params(nx, ny, 3))
    g = np.random.default_rng(5).normal(size=26 * nx * ny)
    p = kpm.KPM_FP32 if prec == "fp32" else kpm.KPM_FP64
    a, _ = _gpu_grad(K, model, fields, ab, M, p, g, 0.7, bw=64, ckpt=7)
    b, _ = _gpu_grad(K, model, fields, ab, M, p, g, 0.7, bw=64, ckpt=7)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- regenerating backward sweep
@pytest.mark.parametrize("nx,ny,M,bw,prec", [(4, 4, 24, 0, 0), (7, 4, 64, 13, 0), (12, 8, 128, 0, 1),
                                              (18, 10, 96, 40, 1)])
def test_regenerate_matches_oracle(K, nx, ny, M, bw, prec):
    """ckpt_every = KPM_REGENERATE (alpha_m rebuilt by the recursion run
    backwards from its last two vectors, Eq. alpha): the oracle's
    Daleckii-Krein gradient to 1e-10 (FP64) and 2e-5 relative (FP32)."""
    kpm, _ = K
    w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), M)
    p = inputs.vortex_seed(w) if prec == 1 else inputs.random_params(nx, ny, 3)
    model, phi, params, fields, ab = _prep(K, nx, ny, p)
    rng = np.random.default_rng(nx + ny)
    g_obs, g_om = rng.normal(size=26 * nx * ny), 0.4
    # a fresh context: its scratch holds exactly what this mode asks for
    fresh = kpm.kpm_create(0)
    try:
        out = torch.empty(26 * nx * ny, dtype=torch.float64, device="cuda")
        kpm.kpm_backward(fresh, model, kpm.make_opts(M, prec, bw), fields, ab, dev(g_obs), g_om, out,
                         ckpt_every=kpm.KPM_REGENERATE)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    finally:
        kpm.kpm_destroy(fresh)
    ref = adjoint.vjp_dense(rmft.Model(nx, ny), fields.cpu().numpy(), *ab.cpu().numpy(), M, g_obs, g_om)
    tol = 1e-10 if prec == 0 else 2e-5
    assert np.max(np.abs(got - ref)) < tol * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", [0, 1])
def test_regenerate_from_kept_tail(K, prec):
    """A kpm_observables with KPM_FLAG_KEEP_TAIL leaves the last two vectors
    of every slab; the regenerating backward pass on the same fields then runs
    no forward sweep and gives the same bits as with its own sweep; after the
    fields change the tail is not used (the gradient follows the new fields)."""
    kpm, _ = K
    nx, ny, M = 10, 8, 80
    N = nx * ny
    w = inputs.Workload(nx, ny, 0.15, inputs.two_vortex(nx, ny), M, seed=2)
    model, phi, params, fields, ab = _prep(K, nx, ny, inputs.vortex_seed(w))
    ctx = kpm.kpm_create(0)  # fresh scratch, sized by this mode alone
    g = dev(np.random.default_rng(4).normal(size=26 * N))
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    opts = kpm.make_opts(M, prec, 48)
    kpm.kpm_observables(ctx, model, opts, fields, ab, obs)  # no tail
    own = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_backward(ctx, model, opts, fields, ab, g, 0.3, own, ckpt_every=kpm.KPM_REGENERATE)
    kept = kpm.make_opts(M, prec, 48, flags=kpm.KPM_FLAG_KEEP_TAIL)
    obs2 = torch.empty_like(obs)
    kpm.kpm_observables(ctx, model, kept, fields, ab, obs2)
    assert torch.equal(obs, obs2)
    tail = torch.empty_like(own)
    kpm.kpm_backward(ctx, model, opts, fields, ab, g, 0.3, tail, ckpt_every=kpm.KPM_REGENERATE)
    assert torch.equal(own, tail)
    # changed fields after the forward pass: the tail no longer matches
    fields2 = fields.clone()
    fields2[:N] += 0.01
    new = torch.empty_like(own)
    kpm.kpm_backward(ctx, model, opts, fields2, ab, g, 0.3, new, ckpt_every=kpm.KPM_REGENERATE)
    ref = adjoint.vjp_dense(rmft.Model(nx, ny), fields2.cpu().numpy(), *ab.cpu().numpy(), M, g.cpu().numpy(), 0.3)
    tol = 1e-10 if prec == 0 else 2e-5
    assert np.max(np.abs(new.cpu().numpy() - ref)) < tol * max(1.0, np.max(np.abs(ref)))
    kpm.kpm_destroy(ctx)


def test_autograd_regenerates_from_forward_tail(K):
    """The autograd Function keeps the forward pass's tail and regenerates:
    its gradient equals kpm_backward with checkpoints (FP64, 1e-12)."""
    kpm, ctx = K
    from paper_2212_05685_gb300 import autograd
    nx, ny, M = 8, 6, 64
    N = nx * ny
    model, phi, params, fields, ab = _prep(K, nx, ny, inputs.random_params(nx, ny, 8))
    opts = kpm.make_opts(M, kpm.KPM_FP64)
    f = fields.clone().requires_grad_(True)
    obs, om = autograd.observables(ctx, model, opts, f, ab)
    wgt = dev(np.random.default_rng(6).normal(size=26 * N))
    ((obs * wgt).sum() + 0.2 * om.sum()).backward()
    ref = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_backward(ctx, model, opts, fields, ab, wgt, 0.2, ref, ckpt_every=8)
    assert float((f.grad - ref).abs().max()) < 1e-12 * max(1.0, float(ref.abs().max()))
