"""The recursion autotuner picks a configuration that fits, is cached per
lattice, and gives the same observables as the default configuration."""
import numpy as np
import pytest

from paper_2212_05685_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nx,ny,prec", [(16, 16, 1), (48, 24, 1), (12, 10, 0)])
def test_autotune_choice_is_valid_and_cached(nx, ny, prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_05685_gb300 import build, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    N = nx * ny
    model = kpm.make_model(nx, ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = torch.tensor(inputs.vortex_seed(inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64)),
                          device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    M = 128
    base = kpm.make_opts(M, prec)
    best, ms = kpm.kpm_autotune(ctx, model, base, fields, ab)
    assert ms >= 0.0  # time per moment from the difference of two trial passes
    assert 1 <= best.block_width <= 2 * N
    assert best.cols_per_block in ((16, 8, 4) if prec == 1 else (8, 4, 2))
    assert best.M == M and best.precision == prec
    again, ms2 = kpm.kpm_autotune(ctx, model, base, fields, ab)
    assert ms2 == -1.0 and again.block_width == best.block_width and again.cols_per_block == best.cols_per_block
    o1 = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    o2 = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, base, fields, ab, o1)
    kpm.kpm_observables(ctx, model, best, fields, ab, o2)
    torch.cuda.synchronize()
    assert float((o1 - o2).abs().max()) < (2e-5 if prec == 1 else 1e-12)
    kpm.kpm_destroy(ctx)
