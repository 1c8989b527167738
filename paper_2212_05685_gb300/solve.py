"""Self-consistency to a tight tolerance (App. A) through rmft_iterate.

The fixed-point loop of readings R1/R2 is slow near a vortex solution: the
density channel must be mixed with a small alpha_n, and linear mixing then
needs of the order of 10^4 iterations for 1e-7 on the 48 x 24 cell.  This
driver runs three phases of the library's loop (every arithmetic step stays
in the C-ABI library; this module only chooses options and stops):

  1. linear mixing in FP32 for `warm` iterations (the transient in which the
     vortex structure forms; Anderson mixing stalls there),
  2. Anderson mixing (reading R4, history `depth`) in FP32 until the residual
     falls below `switch_at` (above the FP32 rounding floor of the
     observables, a few 1e-8),
  3. Anderson mixing with the double-float recursion (FP64-accurate) until
     the residual and the density error are below `tol`.
"""
from __future__ import annotations

import time


def converge(kpm, ctx, model, phi, params, mu_eff, n_target, M, tol=1e-7, warm=500, depth=8, switch_at=1e-6,
             max_fp32=4000, max_df64=400, chunk=200, opts=None):
    """Runs the three phases on (params, mu_eff) in place; returns a record
    with the iterations, wall time and final statistics of each phase."""
    base = opts if opts is not None else kpm.make_opts(M, kpm.KPM_FP32)
    o32 = kpm.kpm_opts.from_buffer_copy(base)
    o32.precision = kpm.KPM_FP32
    odf = kpm.kpm_opts.from_buffer_copy(base)
    odf.precision = kpm.KPM_DF64
    rec = {"tol": tol, "phases": []}

    def phase(name, opts, anderson, limit, stop):
        ro = kpm.make_rmft_opts(n_target, tol=tol, anderson=anderson, sync_every=10)
        done, trace, last = 0, [], None
        t0 = time.perf_counter()
        while done < limit:
            k = min(chunk, limit - done)
            _, st = kpm.rmft_iterate(ctx, model, opts, ro, phi, params, mu_eff, k)
            done += st.iterations
            last = st
            trace.append((done, st.residual, st.density_error))
            if st.converged or st.residual < stop:
                break
        rec["phases"].append({"phase": name, "iterations": done, "s": time.perf_counter() - t0,
                              "residual": last.residual, "density_error": last.density_error, "trace": trace})
        return last

    phase("linear fp32", o32, 0, warm, 0.0)
    st = phase(f"anderson{depth} fp32", o32, depth, max_fp32, switch_at)
    if not st.converged:
        st = phase(f"anderson{depth} df64", odf, depth, max_df64, 0.0)
    rec.update(converged=bool(st.converged), residual=st.residual, density_error=st.density_error, mu=st.mu,
               omega=st.omega, iterations=sum(p["iterations"] for p in rec["phases"]),
               s=sum(p["s"] for p in rec["phases"]))
    return rec
