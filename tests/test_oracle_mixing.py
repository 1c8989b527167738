"""Pins of the Anderson mixing of the oracle (reading R4), independent of the
RMFT map: the linear limit, the exact solution of linear fixed-point problems
(Anderson with a full history is GMRES on (I - J), so it reaches the fixed
point of an affine map of dimension n within n + 1 steps), and agreement of
the RMFT update with `update` when the history is empty."""
import numpy as np

from oracle import rmft
from paper_2212_05685_gb300 import inputs


def test_zero_depth_is_linear_mixing():
    rng = np.random.default_rng(0)
    mix = rmft.Anderson(0)
    x = rng.normal(size=7)
    for _ in range(3):
        f = rng.normal(size=7)
        assert np.array_equal(mix.step(x, f), x + f)


def test_affine_fixed_point_in_n_plus_one_steps():
    """G(x) = A x + b with spectral radius 3 (linear mixing with beta = 1
    diverges): Anderson(m >= n) finds x* = (I - A)^-1 b."""
    rng = np.random.default_rng(1)
    n = 6
    Q = np.linalg.qr(rng.normal(size=(n, n)))[0]
    A = Q @ np.diag([3.0, -2.0, 0.9, 0.5, -0.7, 0.1]) @ Q.T
    b = rng.normal(size=n)
    xs = np.linalg.solve(np.eye(n) - A, b)
    mix = rmft.Anderson(n)
    x = np.zeros(n)
    for k in range(n + 2):
        x = mix.step(x, 0.3 * (A @ x + b - x))
    assert np.max(np.abs(x - xs)) < 1e-8 * np.max(np.abs(xs))


def test_linear_contraction_faster_than_linear_mixing():
    rng = np.random.default_rng(2)
    n = 40
    Q = np.linalg.qr(rng.normal(size=(n, n)))[0]
    A = Q @ np.diag(np.linspace(-0.95, 0.99, n)) @ Q.T
    b = rng.normal(size=n)
    xs = np.linalg.solve(np.eye(n) - A, b)
    lin, acc = np.zeros(n), np.zeros(n)
    mix = rmft.Anderson(16)
    for _ in range(60):
        lin = lin + 0.5 * (A @ lin + b - lin)
        acc = mix.step(acc, 0.5 * (A @ acc + b - acc))
    # 60 steps: linear mixing is still at O(1) error (slowest factor 0.995 per step)
    assert np.max(np.abs(acc - xs)) < 1e-5 * np.max(np.abs(lin - xs))


def test_first_anderson_update_equals_linear_update():
    """Without history the Anderson update is the linear update of readings R1/R2."""
    w = inputs.Workload(6, 4, 0.125, inputs.two_vortex(6, 4), 32)
    p = inputs.vortex_seed(w)
    rng = np.random.default_rng(3)
    obs = p + 0.01 * rng.uniform(-1, 1, size=p.size)
    a = rmft.update(p, obs, w.n_target, 0.2)
    b = rmft.update_anderson(p, obs, w.n_target, 0.2, rmft.Anderson(5))
    assert np.max(np.abs(a[0] - b[0])) < 1e-15
    assert abs(a[1] - b[1]) < 1e-15 and a[2] == b[2] and a[3] == b[3]
