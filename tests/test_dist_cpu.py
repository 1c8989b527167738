"""The N > 1 benchmark path on CPU ranks (gloo, world size 2): every rank
solves its own cell (different seeds, no data-path collective), the job time
is the maximum over ranks and the value counts the units of all ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")
    import bench
    from paper_2212_05685_gb300 import inputs
    w_, r_, l_ = bench.dist_env()
    cell = bench.rank_cell(r_)
    seed_sum = float(np.sum(inputs.vortex_seed(cell)))
    local_time = 1.0 + 0.5 * r_  # the slower rank sets the job time
    dist.barrier()
    t = bench.max_over_ranks(local_time, w_, "cpu")
    v = bench.job_value(w_, 3, cell.dim * cell.M, t)
    gathered = [None] * w_
    dist.all_gather_object(gathered, (r_, l_, cell.seed, seed_sum, t, v))
    if r_ == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    res = sorted(q.get())
    (r0, l0, s0, sum0, t0, v0), (r1, l1, s1, sum1, t1, v1) = res
    assert (r0, r1) == (0, 1) and (l0, l1) == (0, 1)
    assert s0 != s1 and sum0 != sum1          # independent cells
    assert t0 == t1 == 1.5                     # max over ranks
    assert v0 == v1 == pytest.approx(2 * 3 * 20000 * 2048 / 1.5)
