"""kpm_observables_noalloc: the KPM pass for callers that cannot allocate.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator (a pre-sized arena that forbids outside allocations), or they run
where the implicit synchronisation of cudaMalloc/cudaFree is not affordable.
The allocation-free entry point keeps its intermediates in a fixed 48 MiB
device array of the library.  This file checks, through the C ABI, that two
calls in a row reproduce the context-based kpm_observables within the parity
tolerances (FP64 1e-10, FP32 2e-5), on a lattice whose recursion slabs do not
fit the array at once (so the entry point narrows them), that on a small
lattice both calls agree with the CPU oracle's spectral KPM (App. B) within
the same tolerances, and that oversized problems, host buffers and negative
slab widths are refused.  It runs last (file name) so that a
failure here never hides the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from oracle import bdg, kpm as okpm, rmft

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_05685_gb300 import build, inputs, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    yield kpm, inputs, ctx
    kpm.kpm_destroy(ctx)


def _fields(kpm, inputs, ctx, nx, ny):
    N = nx * ny
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    w = inputs.Workload(nx, ny, 0.15, inputs.two_vortex(nx, ny), 64, seed=3)
    params = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.1, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    return model, fields, ab


@pytest.mark.parametrize("prec,tol", [(1, 2e-5), (0, 1e-10)])
def test_two_calls_match_context_entry_point(env, prec, tol):
    kpm, inputs, ctx = env
    nx, ny, M = 40, 30, 96          # D = 2400: 2 (FP32) or 4 (FP64) slabs in 48 MiB
    N = nx * ny
    model, fields, ab = _fields(kpm, inputs, ctx, nx, ny)
    opts = kpm.make_opts(M, prec)
    ref = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    ref_om = torch.empty(1, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, opts, fields, ab, ref, ref_om)
    torch.cuda.synchronize()
    for call in range(2):
        out = torch.full((26 * N,), float("nan"), dtype=torch.float64, device="cuda")
        om = torch.empty(1, dtype=torch.float64, device="cuda")
        st = kpm.kpm_observables_noalloc(model, opts, fields, ab, out, om)
        torch.cuda.synchronize()
        assert st == kpm.KPM_OK, f"call {call}: status {st}"
        assert torch.isfinite(out).all()
        assert float((out - ref).abs().max()) < tol, f"call {call}"
        assert float(om.item()) == pytest.approx(float(ref_om.item()), rel=1e-5 if prec == 1 else 1e-12)


def test_refuses_what_does_not_fit_and_host_buffers(env):
    kpm, inputs, ctx = env
    # 400 x 400 sites: the moment accumulators alone (10 complex doubles per
    # unit column, D = 320000) exceed 48 MiB
    big = kpm.make_model(400, 400)
    N = 400 * 400
    f = torch.zeros(26 * N, dtype=torch.float64, device="cuda")
    ab = torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda")
    o = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    assert kpm.kpm_observables_noalloc(big, kpm.make_opts(16, 1), f, ab, o) == kpm.KPM_EINVAL
    model, fields, ab2 = _fields(kpm, inputs, ctx, 6, 4)
    host = np.zeros(26 * 24)
    assert kpm.kpm_observables_noalloc(model, kpm.make_opts(16, 1), fields, ab2, host) == kpm.KPM_EINVAL
    # a valid call still works afterwards
    out = torch.empty(26 * 24, dtype=torch.float64, device="cuda")
    assert kpm.kpm_observables_noalloc(model, kpm.make_opts(16, 1), fields, ab2, out) == kpm.KPM_OK
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()


@pytest.mark.parametrize("prec,tol", [(1, 2e-5), (0, 1e-10)])
def test_two_calls_match_oracle(env, prec, tol):
    kpm, inputs, ctx = env
    nx, ny, M = 10, 8, 64
    N = nx * ny
    model, fields, ab = _fields(kpm, inputs, ctx, nx, ny)
    w = inputs.Workload(nx, ny, 0.15, inputs.two_vortex(nx, ny), 64, seed=3)
    om = rmft.Model(nx, ny)
    f = rmft.fields(om, inputs.vortex_seed(w), 0.1)
    a, b = bdg.gershgorin(om, f)
    F1, omega = okpm.f_spectral(bdg.dense(om, f), a, b, M)
    ref = okpm.observables(om, F1)
    for call in range(2):
        out = torch.full((26 * N,), float("nan"), dtype=torch.float64, device="cuda")
        o = torch.empty(1, dtype=torch.float64, device="cuda")
        assert kpm.kpm_observables_noalloc(model, kpm.make_opts(M, prec), fields, ab, out, o) == kpm.KPM_OK
        torch.cuda.synchronize()
        assert np.max(np.abs(out.cpu().numpy() - ref)) < tol, f"call {call}"
        assert float(o.item()) == pytest.approx(omega, rel=1e-5 if prec == 1 else 1e-11)


def test_refuses_negative_widths(env):
    kpm, inputs, ctx = env
    model, fields, ab = _fields(kpm, inputs, ctx, 6, 4)
    out = torch.empty(26 * 24, dtype=torch.float64, device="cuda")
    assert kpm.kpm_observables_noalloc(model, kpm.make_opts(16, 1, block_width=-1), fields, ab, out) == kpm.KPM_EINVAL
    assert kpm.kpm_observables_noalloc(model, kpm.make_opts(16, 1, cols_per_block=-2), fields, ab, out) == \
        kpm.KPM_EINVAL
    assert kpm.kpm_observables_noalloc(model, kpm.make_opts(16, 1, site_begin=1, site_end=3), fields, ab, out) == \
        kpm.KPM_EINVAL
