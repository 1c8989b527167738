#!/usr/bin/env python
"""Benchmark of the KPM-RMFT hot path on the 100 x 100 two-vortex cell.

One step = one self-consistency iteration of App. A on the 100 x 100 magnetic
cell (10^4 sites, BdG dimension D = 20000, M = 2048 Chebyshev moments, FP32
recursion vectors with FP64 moment sums): fields, spectral bounds,
coefficients, the block Chebyshev recursion over all D unit start vectors,
observable assembly and the mixing update, through the C ABI (`rmft_iterate`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own independent cell (weak
scaling, no data-path collective); rank 0 prints one JSON line.  The
reference arm (`--impl reference`) times the CPU oracle (naive Chebyshev
recursion on unit vectors, FP64) on a bounded sample of the same pass.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KPM vector-moments/s & s per RMFT iteration at 100x100, FP64 vs FP32 at stated error"
UNIT = "vector-moments/s"
WORKLOAD = "100x100 two-vortex magnetic cell + period-8 PDW seed, D=20000, M=2048, all unit start vectors"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--block-width", type=int, default=0)
    ap.add_argument("--cols", type=int, default=0)
    ap.add_argument("--band-rows", type=int, default=0,
                    help="lattice rows per CTA of the one-step recursion (0: the library's choice)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sample-cols", type=int, default=4, help="oracle columns per worker per step")
    ap.add_argument("--error-sites", type=int, default=112,
                    help="sites (two unit columns each) of the FP32-error and CPU-baseline sample")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-ph-half", action="store_true", help="skip the particle-hole half-pass section")
    ap.add_argument("--no-probing", action="store_true", help="skip the probing-estimator section")
    ap.add_argument("--no-ldos", action="store_true", help="skip the LDOS section")
    ap.add_argument("--no-df64", action="store_true", help="skip the double-float recursion section")
    ap.add_argument("--double-step", action="store_true",
                    help="FP32 recursion two steps per launch (default: as the autotuner chooses, else one)")
    ap.add_argument("--profile-probing", action="store_true",
                    help="one probing pass (100x100, p = 10, M = 64) for ncu launch lists, and exit")
    ap.add_argument("--lbfgs-study", action="store_true",
                    help="64x64 fixed-point loop against the L-BFGS driver (field residual vs passes) and exit")
    ap.add_argument("--profile-adjoint", nargs="?", const="small", choices=["small", "full"],
                    help="run the adjoint case used for ncu captures (small, or the benchmarked full pass) and exit")
    ap.add_argument("--fd-study", type=int, nargs="?", const=200, default=None,
                    help="64x64 adjoint against central finite differences on N field components (default 200), and exit")
    ap.add_argument("--fd-forward", choices=["df64", "fp64"], default="df64",
                    help="recursion of the finite-difference forward passes of --fd-study")
    ap.add_argument("--cfg1-study", action="store_true",
                    help="48x24 cell to self-consistency at 1e-7 (solve.converge) against linear mixing alone, and exit")
    ap.add_argument("--profile-batched", action="store_true",
                    help="one batched iteration (4 cells 48x24 and 2 cells 64x32, M=64, FP32) for ncu captures")
    ap.add_argument("--precision", choices=["fp32", "fp64", "df64"], default="fp32",
                    help="recursion of --profile-small")
    ap.add_argument("--profile-small", action="store_true",
                    help="one FP32 pass on the 100x100 cell with 2000-column slabs and M=8, for ncu captures")
    ap.add_argument("--batched-study", action="store_true",
                    help="the batched section alone (32 cells 24x12 .. 64x32, M=1024), and exit")
    ap.add_argument("--width-study", type=int, nargs="?", const=0, default=None,
                    help="per-step recursion rate against the slab width (full and half pass) on the 100x100 cell; "
                         "with a width, one half pass at that width and M=8 for ncu captures")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_cell(rank):
    """The benchmark cell of one rank: the 100x100 workload with its own seed
    (independent problems per GPU, weak scaling, no data-path collective)."""
    import dataclasses
    from paper_2212_05685_gb300 import inputs
    return dataclasses.replace(inputs.CFG2, seed=inputs.CFG2.seed + rank)


def max_over_ranks(x, world, device):
    """Largest value of x over the ranks (the slowest rank sets the job time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, units_per_step, seconds):
    """Whole-job throughput: the units all ranks processed / the job time."""
    return world * steps * units_per_step / seconds


# ----------------------------------------------------------------------------- clocks

FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
          "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
          "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class Clocks:
    """nvidia-smi samples every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        finally:
            os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- oracle sample (CPU)

class OracleSample:
    """The oracle's naive KPM (scipy CSR x unit-vector block, FP64) on a sample
    of the benchmark pass's unit columns, one spawn-started process per host
    core (oracle/pool.py), on the seed Hamiltonian of the benchmark cell."""

    def __init__(self, cols_per_worker, workers=None):
        from oracle import pool
        from paper_2212_05685_gb300 import inputs
        self.w = inputs.CFG2
        self.workers = workers or len(os.sched_getaffinity(0))
        self.cols = cols_per_worker
        self.pool = pool.ColumnPool(self.w.nx, self.w.ny, inputs.vortex_seed(self.w), 0.0, self.w.M, self.workers)
        self.rng = 0

    def step(self):
        D = self.w.dim
        jobs = []
        for k in range(self.workers):
            start = (self.rng * 7919 + k * 1013) % (D - self.cols)
            jobs.append(list(range(start, start + self.cols)))
        self.rng += 1
        dt = self.pool.time_columns(jobs)
        n = self.workers * self.cols
        return dt, n * self.w.M / dt, n

    def sites(self, count):
        """Order parameters of `count` sampled sites (both vortex cores with
        their neighbours, the rest drawn across the cell) from their 2 count
        columns, and the wall time."""
        from oracle import pool
        sites = pool.sample_sites(self.w.nx, self.w.ny, count, self.w.vortices, seed=5)
        n, chi, F, dt = self.pool.site_observables(sites)
        return sites, n, chi, F, dt

    def close(self):
        self.pool.close()


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    samp = OracleSample(args.sample_cols)
    for _ in range(args.warmup):
        samp.step()
    times, cols = [], 0
    for _ in range(args.steps):
        dt, _, n = samp.step()
        times.append(dt)
        cols += n
    samp.close()
    total = sum(times)
    value = cols * samp.w.M / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "nx": 100, "ny": 100, "M": 2048, "D": 20000},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": samp.workers, "kind": "oracle",
                         "sample": f"{samp.workers * args.sample_cols} of 20000 unit columns per step "
                                   f"(naive FP64 Chebyshev recursion, scipy CSR, M=2048)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm

def source_key(text):
    """sha256 prefix of a kernel source without its // comments and blank
    lines: the key of committed ncu counters (a change of comments keeps
    them; the file has no // inside string literals and no block comments)."""
    code = [line.split("//", 1)[0].rstrip() for line in text.splitlines()]
    return hashlib.sha256("\n".join(c for c in code if c.strip()).encode()).hexdigest()[:16]


def kernel_hash():
    return source_key(open(os.path.join(ROOT, "paper_2212_05685_gb300", "csrc", "cheb_kernels.cu")).read())


def measured_traffic(name, kernel_key, ldv):
    """DRAM bytes per launch from the committed ncu summary `name`, if it was
    taken on the current kernel source; scaled to the benchmark's slab width."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha256_16") != kernel_key:
        return None
    return rec["dram_bytes_per_launch"] * ldv / rec["ldv"]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2212_05685_gb300 import build, inputs, kpm
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    kpm.load()

    w = rank_cell(rank)
    N, D, M = w.n_sites, w.dim, w.M
    stream = torch.cuda.current_stream()
    ctx = kpm.kpm_create(local)
    model = kpm.make_model(w.nx, w.ny, w.t, w.tp, w.J, w.flux)
    opts = kpm.make_opts(M, kpm.KPM_FP32, args.block_width, args.cols, band_rows=args.band_rows,
                         flags=kpm.KPM_FLAG_DOUBLE_STEP if args.double_step else 0)
    ropts = kpm.make_rmft_opts(w.n_target, tol=0.0)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p0 = inputs.vortex_seed(w)
    params = torch.tensor(p0, device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")

    # recursion launch configuration: the library's autotuner (slab width,
    # column chunk) on this cell's Hamiltonian, unless fixed on the command line
    tune = None
    if not args.no_autotune and args.block_width == 0 and args.cols == 0 and args.band_rows == 0:
        f0 = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        ab0 = torch.empty(2, dtype=torch.float64, device="cuda")
        kpm.kpm_build_H(ctx, model, phi, params, 0.0, f0)
        kpm.kpm_bounds(ctx, model, f0, 0.01, ab0)
        t0 = time.perf_counter()
        opts, ms_step = kpm.kpm_autotune(ctx, model, opts, f0, ab0)
        tune = {"block_width": opts.block_width, "cols_per_block": opts.cols_per_block, "band_rows": opts.band_rows,
                "trial_ms_per_step": ms_step, "tuning_s": time.perf_counter() - t0}
        del f0, ab0

    # the benchmarked pass on the seed Hamiltonian: its FP32 error is checked
    # against the oracle's columns in the CPU-baseline leg
    seed_pass = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    fs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    abs_ = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fs)
    kpm.kpm_bounds(ctx, model, fs, 0.01, abs_)
    kpm.kpm_observables(ctx, model, opts, fs, abs_, seed_pass)
    del fs, abs_

    for _ in range(args.warmup):
        kpm.rmft_iterate(ctx, model, opts, ropts, phi, params, mu, 1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    rec_ms, rec_bytes, rec_launches, launches, last = 0.0, 0.0, 0, 0, None
    for _ in range(args.steps):
        _, st = kpm.rmft_iterate(ctx, model, opts, ropts, phi, params, mu, 1)
        rec_ms += st.recursion_ms
        rec_bytes += st.recursion_bytes
        rec_launches += st.recursion_launches
        launches += st.kernel_launches
        last = st
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, "cuda")
    value = job_value(world, args.steps, D * M, t)

    # end to end through the public call with pinned host buffers: the step's
    # parameters (and phases) go host->device, the updated parameters and the
    # statistics come back, inside the timed region
    e2e = None
    if not args.no_e2e:
        hp = torch.tensor(p0).pin_memory()
        hphi = phi.cpu().pin_memory()
        hmu = torch.zeros(1, dtype=torch.float64).pin_memory()
        kpm.rmft_iterate(ctx, model, opts, ropts, hphi, hp, hmu, 1)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            kpm.rmft_iterate(ctx, model, opts, ropts, hphi, hp, hmu, 1)
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        e2e = {"value": job_value(world, args.steps, D * M, te), "unit": UNIT,
               "h2d_bytes_per_step": (26 * N + 4 * N + 1) * 8,
               "d2h_bytes_per_step": (26 * N + 1) * 8 + 8 * 8}

    if rank != 0:
        kpm.kpm_destroy(ctx)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel: the recursion, timed live by the
    # library's CUDA events around the step launches of every timed iteration;
    # algorithmic bytes = the slab vectors each launch must stream (double
    # step: read V_{m-1}, V_m, write V_{m+1}, V_{m+2}; single step: read V_m,
    # V_{m-1}, write V_{m+1}; 8 B per complex element), summed by the library
    cb = opts.cols_per_block if opts.cols_per_block > 0 else 16
    width = opts.block_width if 0 < opts.block_width < D else D
    ldv = (width + cb - 1) // cb * cb
    per_launch_s = rec_ms / 1e3 / max(rec_launches, 1)
    alg_bytes = rec_bytes / max(rec_launches, 1)
    vecs_per_launch = alg_bytes / (D * ldv * 8)
    dbl = vecs_per_launch > 3.5
    # single step: chunks of 8 or 16 columns run the TMA-staged kernel
    kname = "cheb_step2_f32_kernel" if dbl else (
        "cheb_step_f32_tma_kernel<%d,1>" % cb if cb >= 8 else "cheb_step_f32_kernel<%d,1>" % cb)
    pk, pk_kind = peaks()
    achieved = rec_bytes / (rec_ms / 1e3) / 1e9
    nslab = 4 if dbl else 2
    # the committed ncu counters were taken on a 2000-column slab (both slab
    # vectors larger than L2); they scale by columns to any slab that is too
    traffic = measured_traffic("cheb_step2_fp32_100x100.json" if dbl else "cheb_step_fp32_100x100.json",
                               kernel_hash(), ldv) if 2 * D * ldv * 8 > 129e6 else None

    # measured FMA rates of the FP64 and FP32 pipes (the ALU-bound rooflines)
    alu = kpm.kpm_measure_peaks(ctx)
    alu_peaks = {"fp64_tflops": alu[0], "fp32_tflops": alu[1], "fp32x2_tflops": alu[2], "sm_mhz": alu[3],
                 "how": "independent FMA chains (8 per thread, 4 x 256 threads per SM), best of 3 launches for each of two operand patterns (shared or per-chain multiplier and addend), "
                        "CUDA events (kpm_measure_peaks)"}
    props = torch.cuda.get_device_properties(0)
    sm_count = props.multi_processor_count
    sm_mhz_run = (clk or {}).get("sm_mhz") or alu[3]

    fp64 = None
    if not args.no_fp64:
        # FP64 recursion at M = 128, scaled to M = 2048 (cost is linear in M)
        Ms = 128
        fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        ab = torch.empty(2, dtype=torch.float64, device="cuda")
        obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
        kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
        o64 = kpm.make_opts(Ms, kpm.KPM_FP64)
        kpm.kpm_observables(ctx, model, o64, fields, ab, obs)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        kpm.kpm_observables(ctx, model, o64, fields, ab, obs)
        a1.record(stream)
        torch.cuda.synchronize()
        t64 = a0.elapsed_time(a1) / 1e3 * (M - 1) / (Ms - 1)
        # FP64 step: 13 complex multiply-adds and one complex subtraction per
        # row-column (106 flops) against the measured FP64 FMA rate
        fp64_tflops = 106.0 * D * D * (M - 1) / t64 / 1e12
        # one RMFT iteration = the pass + the O(N) work around it, taken from
        # the FP32 iteration (its time minus its recursion steps)
        other = t / args.steps - rec_ms / 1e3 / args.steps
        fp64 = {"s_per_pass": t64, "s_per_rmft_iteration": t64 + other, "vector_moments_per_s": D * M / t64,
                "roofline": {"bound": "alu", "achieved": fp64_tflops, "peak": alu[0], "unit": "TFLOP/s",
                             "frac": fp64_tflops / alu[0], "peak_kind": "measured FP64 FMA rate (kpm_measure_peaks)",
                             "nominal_peak": 1.25},
                "sample": f"FP64 pass at M={Ms} on the same cell, scaled by (M-1)/({Ms}-1): every step does the "
                          f"same work, so the pass time is linear in M",
                "fp32_speedup": (t64 + other) / (t / args.steps)}

    # double-float recursion (FP64-accurate, FP32 pipes) at M = 128, scaled
    # to M = 2048 like the FP64 line; its error against FP64 is in fp32_error
    df64 = None
    if not args.no_df64:
        Ms = 128
        fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        ab = torch.empty(2, dtype=torch.float64, device="cuda")
        obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
        kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
        odf = kpm.make_opts(Ms, kpm.KPM_DF64)
        kpm.kpm_observables(ctx, model, odf, fields, ab, obs)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        kpm.kpm_observables(ctx, model, odf, fields, ab, obs)
        a1.record(stream)
        torch.cuda.synchronize()
        tdf = a0.elapsed_time(a1) / 1e3 * (M - 1) / (Ms - 1)
        # double-float step: 50 double-float multiply-adds of 12 FP32 operations
        # and two renormalisations of 6 per row-column (an FMA counted once),
        # against the measured FP32 FMA rate in FMAs per second (scalar FMA,
        # the kernel's instruction form)
        df_tops = 612.0 * D * D * (M - 1) / tdf / 1e12
        lane_peak = alu[1] / 2.0
        other = t / args.steps - rec_ms / 1e3 / args.steps
        df64 = {"s_per_pass": tdf, "s_per_rmft_iteration": tdf + other, "vector_moments_per_s": D * M / tdf,
                "roofline": {"bound": "alu", "achieved": df_tops, "peak": lane_peak,
                             "unit": "T FP32 lane operations/s", "frac": df_tops / lane_peak,
                             "peak_kind": "measured FP32 FMA rate (kpm_measure_peaks), FMAs per second",
                             "nominal_peak_at_run_clock": sm_count * 128 * sm_mhz_run * 1e6 / 1e12},
                "fp64_equivalent_tflops": 106.0 * D * D * (M - 1) / tdf / 1e12,
                "fp64_nominal_tflops": 1.25,
                "speedup_vs_fp64": (fp64["s_per_pass"] / tdf) if fp64 else None,
                "sample": f"double-float pass at M={Ms} on the same cell, scaled by (M-1)/({Ms}-1)"}

    # particle-hole half pass on the same cell (paramagnetic singlet sector:
    # n_up = n_dn, chi_up = chi_dn, F_ij = F_ji hold for the seed and are kept)
    ph_half = None
    if not args.no_ph_half:
        oh = kpm.make_opts(M, kpm.KPM_FP32, args.block_width, args.cols, flags=kpm.KPM_FLAG_PH_HALF)
        if not args.no_autotune and args.block_width == 0 and args.cols == 0:
            f0 = torch.empty(26 * N, dtype=torch.float64, device="cuda")
            ab0 = torch.empty(2, dtype=torch.float64, device="cuda")
            kpm.kpm_build_H(ctx, model, phi, params, 0.0, f0)
            kpm.kpm_bounds(ctx, model, f0, 0.01, ab0)
            ab0[1] = 0.0
            oh, _ = kpm.kpm_autotune(ctx, model, oh, f0, ab0)
            del f0, ab0
        ph = torch.tensor(p0, device="cuda")
        mh = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            kpm.rmft_iterate(ctx, model, oh, ropts, phi, ph, mh, 1)
        torch.cuda.synchronize()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        hb, hm = 0.0, 0.0
        for _ in range(args.steps):
            _, sh = kpm.rmft_iterate(ctx, model, oh, ropts, phi, ph, mh, 1)
            hb += sh.recursion_bytes
            hm += sh.recursion_ms
        h1.record(stream)
        torch.cuda.synchronize()
        th = h0.elapsed_time(h1) / 1e3 / args.steps
        ph_half = {"s_per_rmft_iteration": th, "vector_moments_per_s": N * M / th,
                   "speedup_vs_full_pass": (t / args.steps) / th,
                   "recursion_achieved_gbs": hb / (hm / 1e3) / 1e9,
                   "columns": f"{N} of {D} unit columns (j, up); the (j, dn) observables from the particle-hole relation",
                   "flags": oh.flags, "block_width": oh.block_width, "cols_per_block": oh.cols_per_block,
                   "band_rows": oh.band_rows}

    probe = None if args.no_probing else probing_section(kpm, ctx, model, phi, params, M, ropts, p0, args, torch)
    ldos_res = None if args.no_ldos else ldos_section(kpm, ctx, model, phi, torch.tensor(p0, device="cuda"), torch)

    batched = None if args.no_batched else batched_section(kpm, inputs, torch, alu)
    adjoint = None if args.no_adjoint else adjoint_section(kpm, inputs, torch)
    precision = precision_section(kpm, inputs, torch)

    # CPU baseline: the oracle's naive recursion on a sample of this pass's
    # unit columns (the seed Hamiltonian), which also gives the FP32 error of
    # the benchmarked pass at those sites
    cpu, fp32_err = None, None
    if not args.no_cpu_baseline and world == 1:
        import numpy as np
        samp = OracleSample(args.sample_cols)
        sites, rn, rc, rF, dt = samp.sites(args.error_sites)
        samp.close()
        ncol = 2 * len(sites)
        cpu = {"value": ncol * M / dt, "unit": UNIT, "cores": samp.workers, "kind": "oracle",
               "sample": f"{ncol} of {D} unit columns of one pass (the columns of {len(sites)} sampled sites; naive "
                         f"FP64 Chebyshev recursion, scipy CSR, M={M}), {dt:.1f} s"}
        gobs = seed_pass.cpu().numpy()
        gn = gobs[:2 * N].reshape(2, N)[:, sites]
        gc = gobs[2 * N:18 * N].view(np.complex128).reshape(2, 4, N)[:, :, sites]
        gF = gobs[18 * N:].view(np.complex128).reshape(4, N)[:, sites]
        fp32_err = {"cell": "100x100", "M": M, "reference": "oracle naive FP64 recursion on the same columns",
                    "sites": len(sites), "columns": ncol,
                    "sites_include": "both vortex cores and their four neighbours",
                    "max_err_n": float(np.abs(gn - rn).max()), "max_err_chi": float(np.abs(gc - rc).max()),
                    "max_err_F": float(np.abs(gF - rF).max()), "bound": 2e-5}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": w.nx, "ny": w.ny, "D": D, "M": M, "precision": "fp32 vectors, fp64 sums",
                   "slab_width": width, "cols_per_block": cb, "autotune": tune,
                   "s_per_rmft_iteration": t / args.steps, "slab_bytes": nslab * D * ldv * 8,
                   "recursion": "two steps per launch" if dbl else "one step per launch",
                   "l2": ("inputs larger than L2 (%d recursion slabs of %.2f GB)" % (nslab, D * ldv * 8 / 1e9))
                   if D * ldv * 8 > 129e6 else "recursion slabs L2-resident (%.0f MB)" % (nslab * D * ldv * 8 / 1e6),
                   "parallelism": f"{world} independent cells (one per GPU)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                     "kernel": kname, "peak_kind": pk_kind,
                     "alg_bytes_per_launch": alg_bytes, "launch_ms": per_launch_s * 1e3},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "fp64": fp64,
        "df64": df64,
        "fp32_error": fp32_err,
        "fp32_error_48x24": precision,
        "alu_peaks": alu_peaks,
        "ph_half": ph_half,
        "probing": probe,
        "ldos": ldos_res,
        "batched": batched,
        "adjoint": adjoint,
        "residual_last": last.residual if last else None,
    }
    print(json.dumps(line), flush=True)
    kpm.kpm_destroy(ctx)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def batched_section(kpm, inputs, torch, alu=None, iters=3):
    """32 cells of uneven size and doping (shapes 24x12 .. 64x32), M = 1024,
    FP32: one batched graph per iteration (the persistent recursion: every
    moment of every cell in one launch, vectors on chip) vs the cells one
    after another; roofline of the persistent launch against the measured FP32
    FMA rate (its vectors never leave shared memory)."""
    cells = inputs.cfg3_cells(seed=0, count=32)
    M = 1024
    opts = kpm.make_opts(M, kpm.KPM_FP32)
    ctx = kpm.kpm_create(0)
    models, phis, params, ropts = [], [], [], []
    for w in cells:
        m = kpm.make_model(w.nx, w.ny)
        phi = torch.empty(4 * w.n_sites, dtype=torch.float64, device="cuda")
        kpm.kpm_peierls_phases(ctx, m, phi)
        models.append(m)
        phis.append(phi)
        params.append(torch.tensor(inputs.vortex_seed(w), device="cuda"))
        ropts.append(kpm.make_rmft_opts(w.n_target, tol=0.0))
    mu = torch.zeros(len(cells), dtype=torch.float64, device="cuda")
    kpm.rmft_iterate_batched(ctx, models, opts, ropts, phis, params, mu, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, bst = kpm.rmft_iterate_batched(ctx, models, opts, ropts, phis, params, mu, iters)
    torch.cuda.synchronize()
    tb = (time.perf_counter() - t0) / iters
    rec_s = bst[0].recursion_ms / 1e3 / iters
    row_updates = sum(w.dim * w.dim for w in cells) * (M - 1)
    seq_ctx = [kpm.kpm_create(0) for _ in cells]
    mus = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in cells]
    for k in range(len(cells)):
        kpm.rmft_iterate(seq_ctx[k], models[k], opts, ropts[k], phis[k], params[k], mus[k], 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters):
        for k in range(len(cells)):
            kpm.rmft_iterate(seq_ctx[k], models[k], opts, ropts[k], phis[k], params[k], mus[k], 1)
    torch.cuda.synchronize()
    ts = (time.perf_counter() - t0) / iters
    for c in seq_ctx:
        kpm.kpm_destroy(c)
    kpm.kpm_destroy(ctx)
    vm = sum(w.dim for w in cells) * M
    out = {"cells": len(cells), "shapes": sorted({f"{w.nx}x{w.ny}" for w in cells}), "M": M, "precision": "fp32",
           "s_per_iteration": tb, "vector_moments_per_s": vm / tb,
           "sequential_s_per_iteration": ts, "sequential_vector_moments_per_s": vm / ts, "speedup": ts / tb}
    if rec_s > 0:
        # 106 flops per row-column (13 complex multiply-adds, one subtraction)
        tflops = 106.0 * row_updates / rec_s / 1e12
        out["persistent_recursion"] = {
            "s_per_iteration": rec_s, "launches_per_iteration": bst[0].recursion_launches,
            "effective_gbs": 24.0 * row_updates / rec_s / 1e9,
            "effective_note": "24 B per row-column (read V_m, V_m-1, write V_m+1) as if streamed; the vectors stay "
                              "in shared memory",
            "roofline": {"bound": "alu", "achieved": tflops, "peak": alu[1] if alu else None, "unit": "TFLOP/s",
                         "frac": tflops / alu[1] if alu else None,
                         "peak_kind": "measured FP32 FMA rate (kpm_measure_peaks)"}}
    return out


def probing_section(kpm, ctx, model, phi, params, M, ropts, p0, args, torch):
    """The paper's estimator (App. B): R = 2 p^2 coloured random-phase probing
    vectors instead of all D unit vectors.  Per p: seconds per pass and per RMFT
    iteration, and the largest error of each observable against the exact
    (all-unit-vector) FP32 pass on the same Hamiltonian."""
    N = model.nx * model.ny
    D = 2 * N
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    exact = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, kpm.make_opts(M, kpm.KPM_FP32), fields, ab, exact)
    est = torch.empty_like(exact)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    rows = []
    for p in (5, 10, 20, 25):
        o = kpm.make_opts(M, kpm.KPM_FP32, probe_p=p, probe_seed=1)
        o, _ = kpm.kpm_autotune(ctx, model, o, fields, ab)  # slab of R columns: its own launch shape
        kpm.kpm_observables(ctx, model, o, fields, ab, est)
        torch.cuda.synchronize()
        ev[0].record()
        kpm.kpm_observables(ctx, model, o, fields, ab, est)
        ev[1].record()
        torch.cuda.synchronize()
        t_pass = ev[0].elapsed_time(ev[1]) / 1e3
        d = (est - exact).abs()
        # RMFT iterations with the estimator (fresh seed parameters)
        pp = torch.tensor(p0, device="cuda")
        mu = torch.zeros(1, dtype=torch.float64, device="cuda")
        kpm.rmft_iterate(ctx, model, o, ropts, phi, pp, mu, 1)
        torch.cuda.synchronize()
        ev[0].record()
        kpm.rmft_iterate(ctx, model, o, ropts, phi, pp, mu, args.steps)
        ev[1].record()
        torch.cuda.synchronize()
        rows.append({"p": p, "R": 2 * p * p, "s_per_pass": t_pass, "cols_per_block": o.cols_per_block,
                     "band_rows": o.band_rows, "two_steps_per_launch": bool(o.flags & kpm.KPM_FLAG_DOUBLE_STEP),
                     "s_per_rmft_iteration": ev[0].elapsed_time(ev[1]) / 1e3 / args.steps,
                     "max_err_n": float(d[:2 * N].max()), "max_err_chi": float(d[2 * N:18 * N].max()),
                     "max_err_F": float(d[18 * N:].max())})
    return {"estimator": "R = 2 p^2 probing vectors, colour alpha + 2((x mod p) + p (y mod p)), SplitMix64 phases",
            "reference": f"exact FP32 pass over all {D} unit vectors", "M": M, "rows": rows}


def ldos_section(kpm, ctx, model, phi, params, torch):
    """LDOS of the 100x100 cell at the seed parameters (App. C): 201
    frequencies in [-0.5 t, 0.5 t], Gamma = 0.25 |w| + 3e-4 t, Gutzwiller
    weights; diagonal moments by probing (p = 10, R = 200) at M = 65536 (the
    resolvent series converges like |w|^M, |w| ~ 1 - Gamma/a at the band
    centre, so M must exceed a few a / Gamma_0)."""
    import numpy as np
    N = model.nx * model.ny
    M, p, nw = 65536, 10, 201
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    omega = np.linspace(-0.5, 0.5, nw)
    out = torch.empty(2 * nw * N, dtype=torch.float64, device="cuda")
    opts = kpm.make_opts(M, kpm.KPM_FP32, probe_p=p, probe_seed=1)
    kpm.kpm_ldos(ctx, model, opts, fields, ab, params, omega, out)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    kpm.kpm_ldos(ctx, model, opts, fields, ab, params, omega, out)
    ev[1].record()
    torch.cuda.synchronize()
    a = float(ab[0])
    # truncation |w|^M at the band centre, w = z - sqrt(z^2 - 1), z = i Gamma_0 / a
    z = 1j * 3e-4 / a
    wc = abs(z - np.sqrt(z * z - 1))
    tot = out.view(2, nw, N).sum(0)
    return {"cell": "100x100", "n_omega": nw, "omega_range_t": [-0.5, 0.5], "gamma": "0.25|w| + 3e-4",
            "M": M, "moments": f"probing p={p} (R={2 * p * p})", "precision": "fp32 recursion, fp64 moments and GEMM",
            "s_total": ev[0].elapsed_time(ev[1]) / 1e3, "truncation_at_w0": wc ** M,
            "mean_ldos_at_w0": float(tot[nw // 2].mean())}


def precision_section(kpm, inputs, torch):
    """FP32 recursion error against the FP64 recursion, per observable, on the
    48 x 24 cell (D = 2304, M = 1024) at its seeded order parameters."""
    w = inputs.CFG1
    N = w.n_sites
    ctx = kpm.kpm_create(0)
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 1.7, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    out = {}
    for name, prec in (("fp64", kpm.KPM_FP64), ("fp32", kpm.KPM_FP32), ("df64", kpm.KPM_DF64)):
        obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        kpm.kpm_observables(ctx, model, kpm.make_opts(w.M, prec), fields, ab, obs)
        out[name] = obs
    torch.cuda.synchronize()
    d = (out["fp32"] - out["fp64"]).abs()
    e = (out["df64"] - out["fp64"]).abs()
    kpm.kpm_destroy(ctx)
    return {"cell": "48x24", "M": w.M, "max_err_n": float(d[:2 * N].max()), "max_err_chi": float(d[2 * N:18 * N].max()),
            "max_err_F": float(d[18 * N:].max()), "bound": 2e-5,
            "df64_max_err": float(e.max()), "df64_bound": 1e-10}


def adjoint_section(kpm, inputs, torch):
    """64x64 cell, M = 1024, FP32, checkpoints every 32 moments: backward
    time as a multiple of the forward pass."""
    w = inputs.CFG4
    N, M = w.n_sites, w.M
    ctx = kpm.kpm_create(0)
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    opts = kpm.make_opts(M, kpm.KPM_FP32)
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    g = torch.ones(26 * N, dtype=torch.float64, device="cuda")
    out = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_observables(ctx, model, opts, fields, ab, obs)
    kpm.kpm_backward(ctx, model, opts, fields, ab, g, 1.0, out, ckpt_every=32)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    kpm.kpm_observables(ctx, model, opts, fields, ab, obs)
    e[1].record()
    kpm.kpm_backward(ctx, model, opts, fields, ab, g, 1.0, out, ckpt_every=32)
    e[2].record()
    torch.cuda.synchronize()
    tf, tb = e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / 1e3
    # every alpha_m stored (no segment recompute): M slab vectors, here under a
    # 160 GiB scratch budget (the GPU's HBM holds it)
    free, _ = torch.cuda.mem_get_info()
    store_all = None
    if free > 200 * 2 ** 30:
        kpm.kpm_set_scratch_budget(ctx, 160 * 2 ** 30)
        kpm.kpm_backward(ctx, model, opts, fields, ab, g, 1.0, out, ckpt_every=M)
        torch.cuda.synchronize()
        e[1].record()
        kpm.kpm_backward(ctx, model, opts, fields, ab, g, 1.0, out, ckpt_every=M)
        e[2].record()
        torch.cuda.synchronize()
        ts = e[1].elapsed_time(e[2]) / 1e3
        store_all = {"ckpt_every": M, "scratch_budget_gib": 160, "backward_s": ts, "backward_over_forward": ts / tf}
    # regenerating backward pass (the recursion run backwards from the last two
    # vectors): after a forward pass that keeps them (the autograd path), and
    # with its own forward sweep; default scratch budget
    kpm.kpm_set_scratch_budget(ctx, 24 * 2 ** 30)
    kept = kpm.make_opts(M, kpm.KPM_FP32, flags=kpm.KPM_FLAG_KEEP_TAIL)
    kpm.kpm_observables(ctx, model, kept, fields, ab, obs)
    kpm.kpm_backward(ctx, model, opts, fields, ab, g, 1.0, out, ckpt_every=kpm.KPM_REGENERATE)
    torch.cuda.synchronize()
    e[0].record()
    kpm.kpm_observables(ctx, model, kept, fields, ab, obs)
    e[1].record()
    kpm.kpm_backward(ctx, model, opts, fields, ab, g, 1.0, out, ckpt_every=kpm.KPM_REGENERATE)
    e[2].record()
    torch.cuda.synchronize()
    tfk, tbr = e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / 1e3
    kpm.kpm_observables(ctx, model, opts, fields, ab, obs)  # drops the tail
    torch.cuda.synchronize()
    e[1].record()
    kpm.kpm_backward(ctx, model, opts, fields, ab, g, 1.0, out, ckpt_every=kpm.KPM_REGENERATE)
    e[2].record()
    torch.cuda.synchronize()
    tbs = e[1].elapsed_time(e[2]) / 1e3
    regenerate = {"forward_keep_tail_s": tfk, "backward_s": tbr, "backward_over_forward": tbr / tf,
                  "backward_with_own_sweep_s": tbs, "backward_with_own_sweep_over_forward": tbs / tf,
                  "note": "alpha_m regenerated by the recursion run backwards from the forward pass's last two "
                          "vectors (no checkpoints, 4 slab vectors of scratch)"}
    kpm.kpm_destroy(ctx)
    return {"cell": "64x64", "M": M, "ckpt_every": 32, "precision": "fp32", "forward_s": tf, "backward_s": tb,
            "backward_over_forward": tb / tf, "store_all": store_all, "regenerate": regenerate}


def lbfgs_study(warm=50, steps_fp=250, iters_lbfgs=40):
    """The 64x64 adjoint cell (M = 1024, FP32): from the state of `warm`
    fixed-point iterations on the vortex seed, the fixed-point loop and the
    L-BFGS driver over the effective fields (driven by kpm_backward, chemical
    potential held at the warm state's) as field-space residual against KPM
    passes (a backward pass counted as one pass) and wall time."""
    import torch
    from paper_2212_05685_gb300 import build, inputs, kpm, lbfgs
    build.build()
    w = inputs.CFG4
    N, M = w.n_sites, w.M
    ctx = kpm.kpm_create(0)
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p0 = torch.tensor(inputs.vortex_seed(w), device="cuda")
    opts = kpm.make_opts(M, kpm.KPM_FP32)
    ropts = kpm.make_rmft_opts(w.n_target, tol=0.0)
    t0 = time.perf_counter()
    p = p0.clone()
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    _, st = kpm.rmft_iterate(ctx, model, opts, ropts, phi, p, mu, warm)
    p_warm, mu_warm = p.clone(), st.mu
    th = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, p, st.mu, th)
    r_warm = lbfgs.FieldProblem(ctx, model, opts, phi, st.mu, th).residual(th)
    fp_trace = [(0, r_warm, st.residual)]
    done = 0
    while done < steps_fp:
        _, st = kpm.rmft_iterate(ctx, model, opts, ropts, phi, p, mu, 25)
        done += 25
        kpm.kpm_build_H(ctx, model, phi, p, st.mu, th)
        prob = lbfgs.FieldProblem(ctx, model, opts, phi, st.mu, th)
        fp_trace.append((done, prob.residual(th), st.residual))
    t_fp = time.perf_counter() - t0
    t0 = time.perf_counter()
    lb_trace = []
    _, _, info = lbfgs.rmft_lbfgs(ctx, model, opts, phi, p_warm, mu_warm, max_iter=iters_lbfgs, tol=0.0,
                                  trace=lb_trace)
    t_lb = time.perf_counter() - t0
    kpm.kpm_destroy(ctx)
    out = {"cell": "64x64", "M": M, "precision": "fp32", "warm_start_iterations": warm,
           "warm_field_residual": r_warm,
           "fixed_point": {"trace_iterations_field_residual_param_residual": fp_trace, "wall_s": t_fp},
           "lbfgs": {"trace_passes_field_residual": lb_trace, "wall_s": t_lb, "info": info}}
    print(json.dumps(out), flush=True)
    return 0


def cfg1_study(linear_budget=6000):
    """The 48x24 two-vortex cell (M = 1024) to self-consistency at 1e-7:
    solve.converge (linear FP32 warm-up, Anderson FP32, Anderson with the
    double-float recursion) against linear FP32 mixing alone for
    `linear_budget` iterations; iterations, wall time, residual traces."""
    import torch
    from paper_2212_05685_gb300 import build, inputs, kpm, solve
    build.build()
    w = inputs.CFG1
    N = w.n_sites
    ctx = kpm.kpm_create(0)
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    p = torch.tensor(inputs.vortex_seed(w), device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    rec = solve.converge(kpm, ctx, model, phi, p, mu, w.n_target, w.M, tol=1e-7)
    q = torch.tensor(inputs.vortex_seed(w), device="cuda")
    mq = torch.zeros(1, dtype=torch.float64, device="cuda")
    ro = kpm.make_rmft_opts(w.n_target, tol=1e-7, sync_every=10)
    lin, done, t0 = [], 0, time.perf_counter()
    while done < linear_budget:
        _, st = kpm.rmft_iterate(ctx, model, kpm.make_opts(w.M, kpm.KPM_FP32), ro, phi, q, mq, 250)
        done += st.iterations
        lin.append((done, st.residual, st.density_error))
        if st.converged:
            break
    out = {"cell": "48x24", "M": w.M, "delta": w.delta, "tol": 1e-7, "converge": rec,
           "linear_only": {"iterations": done, "s": time.perf_counter() - t0, "trace": lin,
                           "residual": lin[-1][1], "converged": bool(st.converged)}}
    kpm.kpm_destroy(ctx)
    print(json.dumps(out), flush=True)
    return 0


def fd_study(ncomp=200, h=1e-6, forward="df64"):
    """The 64x64 adjoint workload (M = 1024, L = sum_i (n_i - n_target,i)^2,
    n_target seeded as in the configuration): the FP64 and FP32 gradients of
    kpm_backward (regenerating from the forward pass's tail) against central
    finite differences with step h of FP64-accurate forward passes (the
    double-float recursion, or with forward="fp64" the FP64 one, whose
    rounding noise divided by h is the floor of the comparison) on `ncomp`
    seeded field components, the rescaling (a, b) held fixed."""
    import numpy as np
    import torch
    from paper_2212_05685_gb300 import build, inputs, kpm
    build.build()
    w = inputs.CFG4
    N, M = w.n_sites, w.M
    ctx = kpm.kpm_create(0)
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    nt = torch.tensor(inputs.target_density(w, seed=1), device="cuda")
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")

    def grad(prec):
        kpm.kpm_observables(ctx, model, kpm.make_opts(M, prec, flags=kpm.KPM_FLAG_KEEP_TAIL), fields, ab, obs)
        n = obs[:N] + obs[N:2 * N]
        g = torch.zeros(26 * N, dtype=torch.float64, device="cuda")
        g[:N] = 2 * (n - nt)
        g[N:2 * N] = 2 * (n - nt)
        out = torch.empty(26 * N, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        kpm.kpm_backward(ctx, model, kpm.make_opts(M, prec), fields, ab, g, 0.0, out, ckpt_every=kpm.KPM_REGENERATE)
        torch.cuda.synchronize()
        return out.cpu().numpy(), time.perf_counter() - t0

    g64, t64 = grad(kpm.KPM_FP64)
    g32, t32 = grad(kpm.KPM_FP32)
    odf = kpm.make_opts(M, kpm.KPM_FP64 if forward == "fp64" else kpm.KPM_DF64)

    def L(f):
        kpm.kpm_observables(ctx, model, odf, f, ab, obs)
        n = obs[:N] + obs[N:2 * N]
        return float(((n - nt) ** 2).sum())

    rng = np.random.default_rng(1)
    comps = np.sort(rng.choice(26 * N, size=ncomp, replace=False))
    rows = []
    t0 = time.perf_counter()
    for k in comps:
        f = fields.clone()
        f[int(k)] += h
        lp = L(f)
        f[int(k)] -= 2 * h
        lm = L(f)
        rows.append((int(k), (lp - lm) / (2 * h), float(g64[k]), float(g32[k])))
    tfd = time.perf_counter() - t0
    fd = np.array([r[1] for r in rows])
    a64 = np.array([r[2] for r in rows])
    a32 = np.array([r[3] for r in rows])
    scale = float(np.max(np.abs(g64)))
    big = np.abs(a64) >= 1e-3 * scale
    rel64 = np.abs(fd - a64) / np.maximum(np.abs(a64), 1e-300)
    rel32 = np.abs(fd - a32) / np.maximum(np.abs(a64), 1e-300)
    out = {"cell": "64x64", "M": M, "h": h, "components": int(ncomp), "seed": 1,
           "forward": ("FP64 recursion" if forward == "fp64" else "double-float recursion (FP64-accurate)")
                      + ", a and b fixed",
           "fd_abs_err_median": float(np.median(np.abs(fd - a64))),
           "gradient": "kpm_backward, regenerating from the forward pass's tail",
           "max_abs_grad": scale, "components_above_1e-3_of_max": int(big.sum()),
           "fp64_max_rel_err_above_1e-3": float(rel64[big].max()) if big.any() else None,
           "fp64_max_abs_err_over_max_grad": float(np.max(np.abs(fd - a64)) / scale),
           "fp32_max_rel_err_above_1e-3": float(rel32[big].max()) if big.any() else None,
           "fp32_max_abs_err_over_max_grad": float(np.max(np.abs(fd - a32)) / scale),
           "backward_fp64_s": t64, "backward_fp32_s": t32, "fd_s": tfd,
           "rows_index_fd_fp64_fp32": rows}
    kpm.kpm_destroy(ctx)
    print(json.dumps(out), flush=True)
    return 0


def profile_adjoint(full=False):
    """Adjoint case for ncu: the 64x64 cell, FP32.  Small (default): M = 64,
    checkpoints every 8 moments, slabs of 2048 columns (134 MB per slab
    vector, 3.5 GB of adjoint scratch).  full: the benchmarked backward pass
    (M = 1024, checkpoints every 32, library-chosen slab width), once."""
    import torch
    from paper_2212_05685_gb300 import build, inputs, kpm
    build.build()
    w = inputs.CFG4
    N = w.n_sites
    ctx = kpm.kpm_create(0)
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    g = torch.ones(26 * N, dtype=torch.float64, device="cuda")
    out = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    if full:
        kpm.kpm_backward(ctx, model, kpm.make_opts(w.M, kpm.KPM_FP32), fields, ab, g, 1.0, out, ckpt_every=32)
    else:
        kpm.kpm_backward(ctx, model, kpm.make_opts(64, kpm.KPM_FP32, 2048), fields, ab, g, 1.0, out, ckpt_every=8)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
    kpm.kpm_destroy(ctx)
    print("profile-adjoint done")
    return 0


def profile_probing():
    """Probing pass for ncu launch lists: the benchmark lattice, p = 10
    (R = 200 vectors, an L2-resident slab), M = 64."""
    import torch
    from paper_2212_05685_gb300 import build, inputs, kpm
    build.build()
    w = inputs.CFG2
    N = w.n_sites
    ctx = kpm.kpm_create(0)
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    kpm.kpm_observables(ctx, model, kpm.make_opts(64, kpm.KPM_FP32, probe_p=10, probe_seed=1), fields, ab, obs)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(obs).all())
    kpm.kpm_destroy(ctx)
    print("profile-probing done")
    return 0


def profile_batched():
    """Small batch for ncu: 4 cells of 48x24 and 2 of 64x32, M = 64, FP32,
    one iteration of the batched call (one persistent recursion launch)."""
    import torch
    from paper_2212_05685_gb300 import build, inputs, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    shapes = [(48, 24)] * 4 + [(64, 32)] * 2
    models, phis, params, ropts = [], [], [], []
    for k, (nx, ny) in enumerate(shapes):
        w = inputs.Workload(nx, ny, 0.15, inputs.two_vortex(nx, ny), 64, seed=k)
        m = kpm.make_model(nx, ny)
        phi = torch.empty(4 * w.n_sites, dtype=torch.float64, device="cuda")
        kpm.kpm_peierls_phases(ctx, m, phi)
        models.append(m)
        phis.append(phi)
        params.append(torch.tensor(inputs.vortex_seed(w), device="cuda"))
        ropts.append(kpm.make_rmft_opts(w.n_target, tol=0.0))
    mu = torch.zeros(len(shapes), dtype=torch.float64, device="cuda")
    kpm.rmft_iterate_batched(ctx, models, kpm.make_opts(64, kpm.KPM_FP32), ropts, phis, params, mu, 1)
    torch.cuda.synchronize()
    assert all(bool(torch.isfinite(p).all()) for p in params)
    kpm.kpm_destroy(ctx)
    print("profile-batched done")
    return 0


def profile_small(double_step=False, precision="fp32"):
    """Small case for ncu: the benchmark lattice, slabs of 2000 columns
    (2 x 320 MB, larger than L2), M = 8: seven recursion-step launches per
    slab, in bands of 34 lattice rows (the band height the autotuner picks for
    the benchmark's 20000-column slab, so that a launch reads the same halo
    rows per column).  precision fp64 / df64: the same slabs through the FP64
    or the double-float recursion."""
    import torch
    from paper_2212_05685_gb300 import build, inputs, kpm
    build.build()
    w = inputs.CFG2
    N = w.n_sites
    ctx = kpm.kpm_create(0)
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    prec = {"fp32": kpm.KPM_FP32, "fp64": kpm.KPM_FP64, "df64": kpm.KPM_DF64}[precision]
    kpm.kpm_observables(ctx, model, kpm.make_opts(8, prec, 2000, band_rows=34,
                                                  flags=kpm.KPM_FLAG_DOUBLE_STEP if double_step else 0), fields, ab, obs)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(obs).all())
    kpm.kpm_destroy(ctx)
    print("profile-small done")
    return 0


def width_study(half_width=0, band_rows=0):
    """Per-step rate of the FP32 recursion on the benchmark lattice against the
    slab width, for the full pass and the particle-hole half pass: each
    configuration runs two passes of different order (M = 66 and 194), so the
    difference is the time of 128 steps per slab without the per-slab start
    and gather.  With half_width > 0, one half pass at that width and M = 8
    (for ncu, bands of band_rows lattice rows, 0 = the library's choice)
    instead."""
    import torch
    from paper_2212_05685_gb300 import build, inputs, kpm
    build.build()
    w = inputs.CFG2
    N, D = w.n_sites, w.dim
    ctx = kpm.kpm_create(0)
    model = kpm.make_model(w.nx, w.ny)
    phi = torch.empty(4 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_peierls_phases(ctx, model, phi)
    params = torch.tensor(inputs.vortex_seed(w), device="cuda")
    fields = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    ab = torch.empty(2, dtype=torch.float64, device="cuda")
    obs = torch.empty(26 * N, dtype=torch.float64, device="cuda")
    kpm.kpm_build_H(ctx, model, phi, params, 0.0, fields)
    kpm.kpm_bounds(ctx, model, fields, 0.01, ab)
    ab[1] = 0.0  # the half pass needs the centre at 0; the full pass takes it too
    if half_width:
        kpm.kpm_observables(ctx, model, kpm.make_opts(8, kpm.KPM_FP32, half_width, 16, flags=kpm.KPM_FLAG_PH_HALF,
                                                      band_rows=band_rows), fields, ab, obs)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(obs).all())
        kpm.kpm_destroy(ctx)
        print("width-study half pass done")
        return 0
    stream = torch.cuda.current_stream()
    M1, M2 = 66, 194
    rows = []

    def timed(o):
        kpm.kpm_observables(ctx, model, o, fields, ab, obs)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        best = 1e30
        for _ in range(2):
            e0.record(stream)
            kpm.kpm_observables(ctx, model, o, fields, ab, obs)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return best

    configs = []
    for half, ncols, widths in ((0, D, (20000, 10000, 4000, 2000)), (1, D // 2, (10000, 5000, 2500))):
        for width in widths:
            configs.append((half, 0, ncols, width, kpm.KPM_FLAG_DOUBLE_STEP, 0))
            for band in (0, 10, 20, 25, 34, 50, 100):
                configs.append((half, 0, ncols, width, 0, band))
    for band in (0, 3, 5, 9, 10, 12):
        configs.append((0, 10, 2 * 10 * 10, 2 * 10 * 10, 0, band))
    for half, probe, ncols, width, dbl, band in configs:
        flags = dbl | (kpm.KPM_FLAG_PH_HALF if half else 0)
        t1 = timed(kpm.make_opts(M1, kpm.KPM_FP32, width, 16, flags=flags, probe_p=probe, band_rows=band))
        t2 = timed(kpm.make_opts(M2, kpm.KPM_FP32, width, 16, flags=flags, probe_p=probe, band_rows=band))
        ldv = (width + 15) // 16 * 16
        nslab = -(-ncols // width)
        step = (t2 - t1) / (nslab * (M2 - M1))
        over = (t1 - nslab * (M1 - 1) * step) / nslab
        gbs = 3 * D * ldv * 8 / step / 1e9
        rows.append({"pass": "probing p=10" if probe else ("half" if half else "full"), "width": width,
                     "two_steps_per_launch": bool(dbl), "band_rows": band, "slabs": nslab,
                     "ms_per_step": step * 1e3, "stream_gbs": gbs, "ms_start_gather_per_slab": over * 1e3,
                     "s_per_pass_M2048": nslab * (over + 2047 * step)})
    print(json.dumps({"study": "slab width and band height", "cell": "100x100", "cols_per_block": 16,
                      "M": [M1, M2], "bytes_per_step": "3 D ldv 8 (read V_m, V_m-1, write V_m+1)",
                      "band_rows": "0 = library default", "rows": rows}), flush=True)
    kpm.kpm_destroy(ctx)
    return 0


def batched_study():
    """The batched section alone (32-cell mix, M = 1024), with the measured
    FMA rates for its roofline."""
    import torch
    from paper_2212_05685_gb300 import build, inputs, kpm
    build.build()
    ctx = kpm.kpm_create(0)
    alu = kpm.kpm_measure_peaks(ctx)
    kpm.kpm_destroy(ctx)
    print(json.dumps({"study": "batched", "batched": batched_section(kpm, inputs, torch, alu)}), flush=True)
    return 0


def main():
    args = parse()
    if args.batched_study:
        return batched_study()
    if args.width_study is not None:
        return width_study(args.width_study, args.band_rows)
    if args.profile_small:
        return profile_small(args.double_step, args.precision)
    if args.profile_batched:
        return profile_batched()
    if args.profile_probing:
        return profile_probing()
    if args.lbfgs_study:
        return lbfgs_study()
    if args.cfg1_study:
        return cfg1_study()
    if args.fd_study is not None:
        return fd_study(args.fd_study, forward=args.fd_forward)
    if args.profile_adjoint:
        return profile_adjoint(args.profile_adjoint == "full")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
