"""kpm_sync_status: the device fault word of the FP32 recursion reads clean
after ordinary FP32 and FP64 passes (the TMA copies of every launch landed
within their bounded waits)."""
import numpy as np
import pytest

from paper_2212_05685_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_sync_status_clean_after_passes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_05685_gb300 import build, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    try:
        nx, ny = 24, 12
        N = nx * ny
        model = kpm.make_model(nx, ny)
        phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
        kpm.kpm_peierls_phases(ctx, model, phi)
        w = inputs.Workload(nx, ny, 0.125, inputs.two_vortex(nx, ny), 64)
        fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        kpm.kpm_build_H(ctx, model, phi, torch.tensor(inputs.vortex_seed(w), device="cuda"), 0.0, fields)
        ab = torch.empty(2, dtype=torch.float64, device="cuda")
        kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
        obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        for prec in (kpm.KPM_FP32, kpm.KPM_FP64):
            kpm.kpm_observables(ctx, model, kpm.make_opts(64, prec), fields, ab, obs)
            assert kpm.kpm_sync_status(ctx) == kpm.KPM_OK
            assert bool(torch.isfinite(obs).all())
    finally:
        kpm.kpm_destroy(ctx)
