"""Self-consistency of one cell with the KPM pass sharded by sites over ranks.

Every unit start vector of the KPM pass is an independent recursion (App. B,
Eq. alpha), and the columns (j, up), (j, dn) give exactly the order parameters
of site j (readings N2, N3).  A cell therefore shards without any exchange
inside the pass: rank r propagates the unit columns of a contiguous range of
sites and writes the order parameters of those sites (zero elsewhere).  One
iteration of App. A's loop is then

  1. prepare   fields, spectral bounds and mu from the parameters (replicated:
               every rank holds the same parameters and does the same O(N) work)
  2. pass      kpm_observables over the rank's sites
  3. merge     one all-reduce (sum) of [obs (26 N), Omega part]: every entry has
               exactly one non-zero contribution, so the merged obs equal the
               single-rank pass bit for bit (Omega to rounding)
  4. update    the mixing update from the merged obs (replicated, identical on
               every rank), then an all-reduce (max) of the residual and of
               |density error| as a consistency check of the replicas.

The gradient of a loss of the observables (kpm_backward) shards the same way:
each rank back-propagates through its own columns and the field-shaped
gradients are summed with one all-reduce.

Arithmetic runs in the backend (the C-ABI library on a GPU); this module only
partitions, calls and merges.  The communicator is torch.distributed (NCCL
between GPUs, gloo on CPU ranks) or None for one rank.
"""
from __future__ import annotations

from dataclasses import dataclass


def site_partition(n_sites: int, world: int, rank: int):
    """Contiguous site range [begin, end) of `rank`: sizes differ by at most one."""
    if not (0 <= rank < world) or n_sites < world:
        raise ValueError("need 0 <= rank < world <= n_sites")
    q, r = divmod(n_sites, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


class Comm:
    """Sum and max all-reduces over torch.distributed (or nothing for one rank)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0

    def sum_(self, t):
        if self.dist and self.world > 1:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def max_(self, t):
        if self.dist and self.world > 1:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return t


@dataclass
class IterStats:
    residual: float
    density_error: float
    mu: float
    omega: float
    a: float
    b: float


class DeviceBackend:
    """The C-ABI library on this rank's GPU: rmft_prepare, kpm_observables over
    a site range, rmft_update.  params (26 N) and mu_eff (1) are CUDA float64
    tensors, updated in place."""

    def __init__(self, ctx, model, opts, ropts, phi, params, mu_eff):
        import torch
        from . import kpm
        self.kpm, self.torch = kpm, torch
        self.ctx, self.model, self.opts, self.ropts = ctx, model, opts, ropts
        self.phi, self.params, self.mu_eff = phi, params, mu_eff
        N = model.nx * model.ny
        dev = params.device
        self.N = N
        self.fields = torch.empty(26 * N, dtype=torch.float64, device=dev)
        self.ab = torch.empty(2, dtype=torch.float64, device=dev)
        self.mu = torch.empty(1, dtype=torch.float64, device=dev)
        self.buf = torch.empty(26 * N + 1, dtype=torch.float64, device=dev)  # obs | Omega
        self.stats = torch.empty(2, dtype=torch.float64, device=dev)

    def prepare(self):
        self.kpm.rmft_prepare(self.ctx, self.model, self.opts, self.phi, self.params, self.mu_eff, self.fields,
                              self.ab, self.mu)

    def observables(self, begin, end):
        """[obs of sites begin..end-1, zero elsewhere | their part of Omega]."""
        o = self.kpm.kpm_opts.from_buffer_copy(self.opts)
        o.site_begin, o.site_end = begin, end
        obs = self.buf[:26 * self.N]
        om = self.buf[26 * self.N:]
        self.kpm.kpm_observables(self.ctx, self.model, o, self.fields, self.ab, obs, om)
        return self.buf

    def update(self, merged):
        self.kpm.rmft_update(self.ctx, self.model, self.ropts, self.params, merged[:26 * self.N], self.mu_eff,
                             self.stats)
        return self.stats

    def scalars(self, merged):
        self.torch.cuda.current_stream().synchronize()
        ab = self.ab.tolist()
        return IterStats(float(self.stats[0]), float(self.stats[1]), float(self.mu[0]),
                         float(merged[26 * self.N]), ab[0], ab[1])

    def backward(self, begin, end, grad_obs, grad_omega, out, ckpt_every=0):
        o = self.kpm.kpm_opts.from_buffer_copy(self.opts)
        o.site_begin, o.site_end = begin, end
        self.kpm.kpm_backward(self.ctx, self.model, o, self.fields, self.ab, grad_obs, grad_omega, out,
                              ckpt_every=ckpt_every)
        return out


def rmft_iterate_sharded(backend, comm: Comm, n_iter: int, tol: float = 0.0):
    """Up to n_iter iterations of the sharded loop; returns the IterStats of
    the last one and the number done.  Stops when residual and |density
    error| are below tol (identically on every rank)."""
    begin, end = site_partition(backend.N, comm.world, comm.rank)
    last, done = None, 0
    for _ in range(n_iter):
        backend.prepare()
        part = backend.observables(begin, end)
        merged = comm.sum_(part)
        stats = backend.update(merged)
        check = comm.max_(stats.abs().clone())
        last = backend.scalars(merged)
        done += 1
        if not (last.residual == last.residual and last.omega == last.omega):
            raise FloatingPointError("sharded RMFT: non-finite residual or grand potential")
        if not (float(check[0]) == abs(last.residual) and float(check[1]) == abs(last.density_error)):
            raise RuntimeError("sharded RMFT: the replicated updates diverged between ranks")
        if last.residual < tol and abs(last.density_error) < tol:
            break
    return last, done


def backward_sharded(backend, comm: Comm, grad_obs, grad_omega, out, ckpt_every=0):
    """dL/d(fields) of one KPM pass: each rank's columns, summed over ranks
    (backend.prepare() must have run for the current parameters)."""
    begin, end = site_partition(backend.N, comm.world, comm.rank)
    backend.backward(begin, end, grad_obs, grad_omega, out, ckpt_every)
    return comm.sum_(out)
