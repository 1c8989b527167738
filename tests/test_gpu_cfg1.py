"""48 x 24 cell (BdG dimension 2304, M = 1024): per-observable error of the FP32
and FP64 recursions against the FP64 oracle, and one RMFT iteration's residual
and density error against the oracle's update (Sec. II, App. A, B).
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


def test_cfg1_observable_errors(K):
    kpm, ctx = K
    w = inputs.CFG1
    N = w.n_sites
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p = inputs.vortex_seed(w)
    fd = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, torch.tensor(p, device="cuda"), 1.7, fd)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fd, 0.01, ab)
    torch.cuda.synchronize()
    f = fd.cpu().numpy()
    a, b = (float(v) for v in ab.cpu().numpy())
    om = rmft.Model(w.nx, w.ny)
    assert np.max(np.abs(f - rmft.fields(om, p, 1.7))) < 1e-12 * max(1.0, np.max(np.abs(f)))
    F1, omega = okpm.f_spectral(bdg.dense(om, f), a, b, w.M)
    ref = okpm.observables(om, F1)
    assert np.isfinite(ref).all()
    errs = {}
    for prec in (kpm.KPM_FP64, kpm.KPM_FP32):
        obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        o = torch.empty(1, dtype=torch.float64, device="cuda")
        kpm.kpm_observables(ctx, model, kpm.make_opts(w.M, prec), fd, ab, obs, o)
        torch.cuda.synchronize()
        g = obs.cpu().numpy()
        assert np.isfinite(g).all(), (prec, int(np.isnan(g).sum()))
        d = np.abs(g - ref)
        errs[prec] = (d[:2 * N].max(), d[2 * N:18 * N].max(), d[18 * N:].max(), abs(float(o.item()) - omega))
    print("max error vs FP64 oracle (n, chi, F, Omega): fp64", errs[kpm.KPM_FP64], "fp32", errs[kpm.KPM_FP32])
    assert max(errs[kpm.KPM_FP64][:3]) < 1e-10
    assert max(errs[kpm.KPM_FP32][:3]) < 2e-5


def test_cfg1_one_iteration_residual(K):
    kpm, ctx = K
    w = inputs.CFG1
    N = w.n_sites
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p0 = inputs.vortex_seed(w)
    p = torch.tensor(p0, device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    _, st = kpm.rmft_iterate(ctx, model, kpm.make_opts(w.M, kpm.KPM_FP64),
                             kpm.make_rmft_opts(w.n_target, tol=0.0), phi, p, mu, 1)
    om = rmft.Model(w.nx, w.ny)
    f, mu_phys = rmft.shifted_fields(om, p0, 0.0)
    a, b = bdg.gershgorin(om, f)
    F1, omega = okpm.f_spectral(bdg.dense(om, f), a, b, w.M)
    p1, mu1, r, e = rmft.update(p0, okpm.observables(om, F1), w.n_target, 0.0)
    assert st.residual == pytest.approx(r, abs=1e-10)
    assert st.density_error == pytest.approx(e, abs=1e-10)
    assert st.mu == pytest.approx(mu_phys, abs=1e-10)
    assert st.omega == pytest.approx(omega, rel=1e-11)
    assert np.max(np.abs(p.cpu().numpy() - p1)) < 1e-10
    assert float(mu.item()) == pytest.approx(mu1, abs=1e-10)


def test_cfg1_converges_to_1e7(K):
    """The 48 x 24 two-vortex cell at M = 1024 run to self-consistency at
    tol = 1e-7 (max parameter change and density error), through
    solve.converge: 500 linear FP32 iterations, Anderson mixing (reading R4)
    in FP32 to 1e-6, then Anderson with the double-float recursion.  Reading
    R3: the oracle's residual at the GPU's final parameters (one FP64 spectral
    KPM pass and the update of readings R1/R2) is below tol as well."""
    kpm, ctx = K
    from paper_2212_05685_gb300 import solve
    w = inputs.CFG1
    N = w.n_sites
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p = torch.tensor(inputs.vortex_seed(w), device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    rec = solve.converge(kpm, ctx, model, phi, p, mu, w.n_target, w.M, tol=1e-7)
    print({k: v for k, v in rec.items() if k != "phases"},
          [(ph["phase"], ph["iterations"], round(ph["s"], 1), ph["residual"]) for ph in rec["phases"]])
    assert rec["converged"] and rec["residual"] < 1e-7 and abs(rec["density_error"]) < 1e-7
    om = rmft.Model(w.nx, w.ny)
    pf, mf = p.cpu().numpy(), float(mu.item())
    f, _ = rmft.shifted_fields(om, pf, mf)
    a, b = bdg.gershgorin(om, f)
    F1, _ = okpm.f_spectral(bdg.dense(om, f), a, b, w.M)
    _, _, r, e = rmft.update(pf, okpm.observables(om, F1), w.n_target, mf)
    assert r < 1e-7 + 1e-9 and abs(e) < 1e-7 + 1e-9
