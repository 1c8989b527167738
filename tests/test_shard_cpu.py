"""The site-sharded self-consistency loop on CPU ranks (gloo, world size 2).

The driver (paper_2212_05685_gb300/shard.py) partitions the sites, runs the
per-rank pass, merges with one sum all-reduce and applies the replicated
update.  Here the per-rank pass is the oracle's naive recursion (Eq. alpha)
over the rank's unit columns, a stand-in for the device; the merged
parameters after three iterations must equal those of one rank bit for bit
(each merged entry has exactly one non-zero contribution), the grand
potential to rounding, and the sharded backward sum must equal the
one-rank gradient of the oracle's adjoint.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NY, M, ITERS = 6, 4, 32, 3


def test_partition_covers_sites_once():
    from paper_2212_05685_gb300.shard import site_partition
    for n, w in ((24, 2), (25, 4), (7, 7), (10000, 8)):
        ranges = [site_partition(n, w, r) for r in range(w)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        sizes = [e - b for b, e in ranges]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        site_partition(3, 4, 0)


class OracleBackend:
    """Stand-in for the device: the oracle's fields, bounds, naive recursion on
    the range's unit columns and linear update (readings R1, R2)."""

    def __init__(self, w, params):
        from oracle import bdg, rmft
        self.w = w
        self.om = rmft.Model(w.nx, w.ny)
        self.N = self.om.N
        self.params = np.array(params, dtype=np.float64)
        self.mu_eff = 0.0
        self.bdg, self.rmft = bdg, rmft

    def prepare(self):
        self.f, self.mu = self.rmft.shifted_fields(self.om, self.params, self.mu_eff)
        self.a, self.b = self.bdg.gershgorin(self.om, self.f)

    def observables(self, begin, end):
        from oracle import kpm as okpm
        D = 2 * self.N
        cols = np.arange(2 * begin, 2 * end)
        Fc, om = okpm.f_naive(self.bdg.csr(self.om, self.f), self.a, self.b, self.w.M, cols=cols)
        full = np.zeros((D, D), dtype=np.complex128)
        full[:, cols] = Fc
        obs = okpm.observables(self.om, full)
        n, chi, F = self.rmft.split(obs, self.N)
        outside = np.ones(self.N, dtype=bool)
        outside[begin:end] = False
        n[:, outside] = 0.0
        chi[:, :, outside] = 0.0
        F[:, outside] = 0.0
        return torch.tensor(np.concatenate([self.rmft.join(n, chi, F), [om]]))

    def update(self, merged):
        m = merged.numpy()
        self.params, self.mu_eff, r, e = self.rmft.update(self.params, m[:26 * self.N], self.w.n_target,
                                                         self.mu_eff)
        self.r, self.e = r, e
        return torch.tensor([r, e], dtype=torch.float64)

    def scalars(self, merged):
        from paper_2212_05685_gb300.shard import IterStats
        return IterStats(self.r, self.e, self.mu, float(merged[26 * self.N]), self.a, self.b)

    def backward(self, begin, end, grad_obs, grad_omega, out, ckpt_every=0):
        """dL/d(fields) from the rank's columns: the oracle's Daleckii-Krein
        gradient of the loss restricted to the observables of those sites."""
        from oracle import adjoint
        g = np.array(grad_obs.numpy(), copy=True)
        n, chi, F = self.rmft.split(g, self.N)
        outside = np.ones(self.N, dtype=bool)
        outside[begin:end] = False
        n[:, outside] = 0.0
        chi[:, :, outside] = 0.0
        F[:, outside] = 0.0
        # the Omega seed goes to the first rank only: the sum over ranks is the
        # full gradient, the loss being linear in the seeds
        gf = adjoint.vjp_dense(self.om, self.f, self.a, self.b, self.w.M, self.rmft.join(n, chi, F),
                               grad_omega if begin == 0 else 0.0)
        out.copy_(torch.tensor(gf))
        return out


def _workload():
    from paper_2212_05685_gb300 import inputs
    return inputs.Workload(NX, NY, 0.125, inputs.two_vortex(NX, NY), M, seed=4)


def _run(comm):
    from paper_2212_05685_gb300 import inputs, shard
    w = _workload()
    be = OracleBackend(w, inputs.vortex_seed(w))
    stats, done = shard.rmft_iterate_sharded(be, comm, ITERS)
    rng = np.random.default_rng(9)
    g = torch.tensor(rng.uniform(-1, 1, size=26 * be.N))
    out = torch.zeros(26 * be.N, dtype=torch.float64)
    be.prepare()
    shard.backward_sharded(be, comm, g, 0.7, out)
    return be.params, be.mu_eff, stats, done, out.numpy()


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://")
    from paper_2212_05685_gb300 import shard
    comm = shard.Comm()
    res = _run(comm)
    if rank == 0:
        q.put(res)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_rank():
    from paper_2212_05685_gb300 import shard

    class One:
        world, rank = 1, 0

        def sum_(self, t):
            return t

        def max_(self, t):
            return t

    p1, mu1, st1, d1, g1 = _run(One())
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = socket.socket()
    port.bind(("127.0.0.1", 0))
    pnum = port.getsockname()[1]
    port.close()
    procs = [ctx.Process(target=_rank, args=(r, 2, pnum, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    p2, mu2, st2, d2, g2 = q.get()
    assert d1 == d2 == ITERS
    assert np.array_equal(p1, p2)          # merged observables exact, replicated update identical
    assert mu1 == mu2
    assert st1.residual == st2.residual and st1.density_error == st2.density_error
    assert st2.omega == pytest.approx(st1.omega, rel=1e-13)
    assert np.max(np.abs(g2 - g1)) <= 1e-12 * max(1.0, np.max(np.abs(g1)))
    assert shard.site_partition(NX * NY, 2, 1) == (12, 24)
