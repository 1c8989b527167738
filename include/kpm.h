/*
 * kpm.h - C ABI of the GB300 KPM observable engine for the renormalised
 * mean-field (Gutzwiller) vortex solver of arXiv:2212.05685.
 *
 * Every entry point returns an int status (KPM_OK = 0, negative on error; see
 * kpm_strerror) and never throws or aborts across the ABI.  Array arguments
 * are plain pointers owned by the caller; unless stated otherwise they must be
 * device pointers of the context's GPU, 16-byte aligned, and are used
 * asynchronously on `stream` (a cudaStream_t passed as void*, NULL = the
 * legacy default stream).  The context owns only scratch memory (recursion
 * slabs, accumulators, CUDA graphs).
 *
 * Lattice and array layouts (N = nx*ny sites, site i = x + nx*y, periodic):
 *
 *   forward bonds d = 0..3 : i -> i + (+x, +y, +x+y, +x-y)
 *   ordered nn pairs e = 0..3 : i -> i + (+x, +y, -x, -y)
 *
 *   order parameters ("params"/"obs", float64, 26*N):
 *     [0, 2N)     n[s][i]            s = 0 up, 1 down          (Eq. delta, mz)
 *     [2N, 18N)   chi[s][d][i]       complex, interleaved       (Eq. chi)
 *                 chi_{i,i+d,s} = <c^dag_{i s} c_{i+d, s}>
 *     [18N, 26N)  F[e][i]            complex, interleaved       (Eq. pairing)
 *                 F_{i,i+e} = <c_{i up} c_{i+e, dn}>; the paper's
 *                 Delta_{ij up} = F_ij and Delta_{ij dn} = F_ji
 *
 *   effective fields ("fields", float64, 26*N, same layout):
 *     eps[s][i] = dW/dn_{i s},  T[s][d][i] = dW/dchi_{i,i+d,s},
 *     D[e][i] = dW/dF*_{i,i+e}                           (Eqs. Tij, Dij, mu_i)
 *
 *   Nambu matrix (App. B, d_i = (c_{i up}, c^dag_{i dn}), row I = 2i + alpha):
 *     h[(i,0),(i,0)] = eps_{i up},  h[(i,1),(i,1)] = -eps_{i dn},
 *     h[(i,0),(j,0)] = T_{ij up},   h[(i,1),(j,1)] = -conj(T_{ij dn}),
 *     h[(i,0),(j,1)] = -D_{ij},     plus Hermitian conjugates.
 *
 *   Peierls phases ("phi", float64, 4*N): phi[d][i] on the forward bonds,
 *     t_{i,i+d} = t e^{i phi} (d < 2) or t' e^{i phi} (d >= 2)  (Sec. II).
 */
#ifndef KPM_H
#define KPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KPM_OK 0
#define KPM_EINVAL (-1)      /* bad size, null pointer, misaligned or host pointer where a device one is required */
#define KPM_ENOMEM (-2)      /* scratch allocation failed */
#define KPM_ECUDA (-3)       /* a CUDA call failed; kpm_last_error() has the CUDA message */
#define KPM_ENONFINITE (-4)  /* NaN or Inf in an output */
#define KPM_ETIMEDOUT (-5)   /* a bounded device wait of the FP32 recursion expired (kpm_sync_status, rmft_iterate) */
#define KPM_ENOTCONV (-6)    /* rmft_iterate reached n_iter without meeting tol (only if asked to report it) */

#define KPM_FP64 0
#define KPM_FP32 1
#define KPM_DF64 2  /* double-float: FP64-accurate recursion in FP32 hi + lo pairs */

typedef struct kpm_ctx kpm_ctx;

/* t-t'-J model on an nx x ny torus threaded by `flux` quanta hc/e
 * (B = 2 Phi0 / (nx ny) per quantum, App. C).  nx, ny >= 2. */
typedef struct {
  int32_t nx, ny;
  int32_t flux;
  int32_t gutzwiller;   /* 1: Gutzwiller factors of App. A; 0: all g = 1 */
  double t, tp, J;      /* nn hopping, nnn hopping, exchange (paper: 1, -0.3, 0.3) */
} kpm_model;

/* Chebyshev expansion options (App. B). */
typedef struct {
  int32_t M;            /* number of moments, M >= 1 (paper: 1000-2000) */
  int32_t precision;    /* KPM_FP64: FP64 recursion; KPM_FP32: FP32 vectors and
                           coefficients, FP64 moment sums and everything else;
                           KPM_DF64: vectors and coefficients as double-float
                           (hi + lo FP32 pairs, about 48 bits), arithmetic on the
                           FP32 pipes, FP64 everything else (kpm_observables,
                           rmft_iterate, kpm_autotune; refused with KPM_EINVAL by
                           kpm_backward, kpm_ldos, rmft_iterate_batched and
                           kpm_observables_noalloc) */
  int32_t block_width;  /* unit start vectors per slab; 0 = as many as fit the
                           context's scratch budget (kpm_set_scratch_budget) */
  int32_t cols_per_block; /* columns per CTA in the recursion kernel; 0 = default */
  double margin;        /* spectral half-width margin of the Gershgorin rescale (0.01) */
  double temperature;   /* 0: T = 0 step and min(eps, 0) in closed form; T > 0: Fermi
                           function 1/(1 + e^{eps/T}) and grand-potential function
                           -T log(1 + e^{-eps/T}) of the BdG energy eps, coefficients
                           by Chebyshev-Gauss quadrature with 4 M nodes (App. B) */
  int32_t flags;        /* KPM_FLAG_* bits; 0 = defaults */
  int32_t probe_p;      /* 0: all unit start vectors (exact trace).  p >= 2, dividing nx
                           and ny: R = 2 p^2 probing vectors (App. B): Nambu row
                           K = 2 i + alpha of site (x, y) has colour alpha + 2 ((x mod
                           p) + p (y mod p)) and phase xi_K = exp(2 pi i u_K), u_K from
                           SplitMix64 at counter probe_seed * 2^32 + K; column J of
                           F_M(h~) is estimated as conj(xi_J) F_M(h~) r_colour(J).
                           kpm_observables and rmft_iterate only. */
  int32_t probe_seed;   /* phase stream of the probing vectors */
  int32_t site_begin;   /* column range of the pass (App. B: every start vector is an     */
  int32_t site_end;     /* independent recursion): 0, 0 = all sites; else only the unit
                           columns (j, up), (j, dn) of sites j in [site_begin, site_end),
                           0 <= site_begin < site_end <= N, are propagated; obs holds the
                           order parameters of those sites and 0 elsewhere, omega the part
                           of the trace over those columns, so the obs of a partition of the
                           sites sum to the full pass exactly and the omegas to rounding.
                           kpm_observables and kpm_backward (its gradient is then the part
                           from those columns); with probing, KPM_EINVAL. */
  int32_t band_rows;    /* lattice rows per CTA of the one-step recursion kernels (each
                           CTA runs a band of rows of one column chunk); 0 = the
                           library's choice (the best of a wave model: chunks x
                           bands CTAs, one per SM, each costing its rows plus
                           two halo rows of one vector), else min(band_rows, ny).  Changes the
                           launch shape only, not the result; kpm_autotune searches
                           it.  Negative: KPM_EINVAL. */
} kpm_opts;

/* kpm_opts.flags: run the FP32 recursion two steps per launch where the
 * lattice allows it (default: one step per launch; both give the same bits;
 * kpm_autotune picks the faster) */
#define KPM_FLAG_DOUBLE_STEP 1
/* kpm_opts.flags: particle-hole half pass.  Only the N unit columns (j, up)
 * are propagated; the spin-down observables and the other half of the grand
 * potential's diagonal follow exactly from F_M(h~) = 1 - U conj(F_M(h~)) U^T,
 * which holds when eps_up = eps_dn, T_up = T_dn and D_ij = D_ji (the
 * paramagnetic singlet sector, where the spectrum is symmetric and b = 0).
 * kpm_observables and rmft_iterate check the fields (deviation <= 1e-12 of the
 * largest field) and that |b| <= 1e-12 a, else KPM_EINVAL; rmft_iterate
 * rescales with b = 0 exactly.  Not accepted by kpm_backward,
 * rmft_iterate_batched and kpm_observables_noalloc (KPM_EINVAL). */
#define KPM_FLAG_PH_HALF 2
/* kpm_opts.flags: kpm_observables keeps the last two recursion vectors of every
 * slab (alpha_{M-2}, alpha_{M-1}; 2 slab vectors per slab of context memory)
 * and a copy of its fields and ab, so that a following kpm_backward with
 * ckpt_every = KPM_REGENERATE on the same fields runs no forward sweep.  FP32
 * or FP64 unit-vector passes (KPM_EINVAL with probing, the half pass or
 * KPM_DF64); any kpm_observables call without the flag drops the tail. */
#define KPM_FLAG_KEEP_TAIL 4

/* kpm_backward ckpt_every: regenerate the forward vectors backwards instead
 * of checkpointing them (see kpm_backward) */
#define KPM_REGENERATE (-1)

/* Self-consistency options (the paper's iteration, readings R1/R2). */
typedef struct {
  double n_target;      /* electrons per site, 1 - delta */
  double alpha;         /* mixing of chi and F (0.5) */
  double alpha_n;       /* mixing of the densities (0.05) */
  double eta;           /* gain of the chemical-potential feedback (0.5) */
  double tol;           /* converged when max |p_new - p| and |<n> - n_target| < tol */
  int32_t paramagnetic; /* 1: keep n_up = n_dn (m = 0 sector) */
  int32_t strict;       /* 1: rmft_iterate returns KPM_ENOTCONV when its n_iter iterations
                           end without meeting tol (stats and params as after the last
                           iteration); 0: KPM_OK, with stats.converged = 0 */
  int32_t anderson;     /* 0: linear mixing (above).  1..16: Anderson (Pulay) mixing over the
                           last `anderson` iterations of this call (history cleared at the
                           start of every call), applied to the parameters and mu_eff with
                           the linear mixings as preconditioner (reading R4) */
  int32_t sync_every;   /* iterations per host read of the residual (0 or 1: every
                           iteration).  k > 1: k iterations are queued between reads; an
                           iteration that meets tol freezes params and mu_eff on the device,
                           so results, stats and iteration counts equal those of k = 1 */
} kpm_rmft_opts;

/* Per-call results of rmft_iterate (host struct, filled before return). */
typedef struct {
  double residual;      /* max |p_new - p| of the last iteration */
  double density_error; /* <n_new> - n_target of the last iteration */
  double mu;            /* Lagrange multiplier mu = mu_eff + <dW/dn|_{mu=0}> */
  double omega;         /* KPM grand potential Omega_M = a tr G_M(h~) of the last pass */
  double a, b;          /* spectral rescale h~ = (h - b)/a of the last pass */
  double recursion_ms;  /* device time of the Chebyshev recursion steps, summed over
                           this call's iterations (CUDA events recorded on the
                           launching stream around the step launches; with sync_every
                           k > 1 the last iteration of each group of k counts k times) */
  double recursion_bytes; /* algorithmic HBM bytes of those launches, summed the same
                           way: slab vectors each launch must read and write
                           (8 B per FP32 / 16 B per FP64 complex element) */
  int32_t iterations;   /* iterations performed by this call */
  int32_t converged;    /* 1 if the last iteration met tol */
  int32_t kernel_launches;    /* kernels of this library launched per iteration */
  int32_t recursion_launches; /* of which recursion-step launches */
} kpm_rmft_stats;

/* Create a context on CUDA device `device`.  Allocates nothing yet. */
int kpm_create(kpm_ctx** out, int device);
/* Free the context and all its scratch.  Synchronises the device. */
int kpm_destroy(kpm_ctx* ctx);
/* Upper bound (bytes) on recursion-slab scratch; default 24 GiB. */
int kpm_set_scratch_budget(kpm_ctx* ctx, uint64_t bytes);
/* Synchronise `stream` (NULL: the legacy default stream) and read the device
 * fault word of the FP32 recursion: KPM_OK; KPM_ETIMEDOUT when one of its
 * bounded waits for its own TMA copies expired (that launch, and every FP32
 * recursion launch of the process after it until the word is cleared, wrote
 * NaN instead of results); KPM_ECUDA for an asynchronous CUDA error or a
 * recursion that found its shared memory misaligned for TMA (outputs NaN as
 * well).  A word that is reported is cleared (after the device is idle), so
 * later launches compute again; the caller decides whether to trust the
 * device further.  rmft_iterate and rmft_iterate_batched read (and clear) the
 * word themselves when an iteration turns non-finite. */
int kpm_sync_status(kpm_ctx* ctx, void* stream);
/* Failure-path test hook (no counterpart in the paper).  The next `count` CTAs
 * of the TMA-staged FP32 recursion step that would issue the copy of their
 * third window row skip that copy and its expected byte count, so nothing is
 * in flight for that slot and the CTA's bounded waits expire: the launch
 * writes NaN and the fault word reads KPM_ETIMEDOUT, with no device fault.
 * wait_limit_s > 0 sets the bounded-wait limit of every later FP32 recursion
 * launch in the process (default 2 s); <= 0 restores the default.  count = 0
 * withdraws outstanding skips.  Synchronises the device. */
int kpm_inject_lost_copy(kpm_ctx* ctx, int count, double wait_limit_s);
/* Measured ALU peaks of the device (no counterpart in the paper; the
 * denominators of the FP64 and double-float rooflines): independent FMA
 * chains, 8 per thread, 4 CTAs of 256 threads per SM, the chains sharing one
 * multiplier/addend pair or each with its own (the better of the two per
 * kind, best of 3 launches each), timed with CUDA events on `stream`.  out[0] = FP64 FMA TFLOP/s (2 flops per FMA), out[1] = FP32 scalar
 * FMA TFLOP/s, out[2] = FP32 packed f32x2 FMA TFLOP/s (4 flops per
 * instruction), out[3] = median SM clock seen by the kernels in MHz (from
 * %clock64 over %globaltimer).  out: host, 4 doubles.  Synchronises `stream`. */
int kpm_measure_peaks(kpm_ctx* ctx, double* out, void* stream);
const char* kpm_strerror(int status);
/* Last error message of this context (static storage of the context). */
const char* kpm_last_error(const kpm_ctx* ctx);

/* Peierls phases of the Landau gauge A = B(0, x) (Sec. II, App. C), with the
 * magnetic-translation phase 2 pi flux y'/ny on bonds crossing the x boundary
 * and straight-line integrals on next-nearest-neighbour bonds.
 * phi: device, 4*N doubles, written. */
int kpm_peierls_phases(kpm_ctx* ctx, const kpm_model* model, double* phi, void* stream);

/* Effective fields of the renormalised functional (App. A, Eqs. Tij, Dij,
 * mu_i): fields = dW/d(params) at chemical potential `mu`.
 * phi: device 4*N; params: device 26*N; fields: device 26*N (written);
 * w_out: device double or NULL; written with W = <H_renorm> - mu sum_i n_i
 * (the constant mu N_e of App. A omitted). */
int kpm_build_H(kpm_ctx* ctx, const kpm_model* model, const double* phi,
                const double* params, double mu, double* fields, double* w_out,
                void* stream);

/* Gershgorin bounds of the Nambu matrix (App. B "shifting and rescaling"):
 * ab[0] = a = (1 + margin)(Emax - Emin)/2, ab[1] = b = (Emax + Emin)/2, with
 * Emax/Emin over rows of h_II +- sum of the moduli of the 12 off-diagonal
 * stencil entries (a = 1 when Emax = Emin).  fields: device; ab: device, 2 doubles. */
int kpm_bounds(kpm_ctx* ctx, const kpm_model* model, const double* fields,
               double margin, double* ab, void* stream);

/* One KPM pass (App. B, Eqs. rho_KPM, F_KPM, alpha) over all D = 2N unit
 * start vectors: obs = order parameters read off F_M(h~)^T = rho with
 * F_M = sum_m (2 - delta_m0) g_m c_m T_m the Jackson-damped T = 0 step at BdG
 * energy 0; omega = a tr G_M(h~) with G_M the damped series of min(x - x0, 0).
 * fields, ab: device (ab as written by kpm_bounds).  obs: device 26*N,
 * written.  omega: device double or NULL.
 * Asynchronous on `stream`.  The FP32 recursion moves its rows by TMA copies
 * that complete on mbarriers; its waits are bounded in time (2 s), and a
 * recursion whose copies never land writes NaN over the rows it owns (and
 * every later FP32 recursion launch of the process does the same), so such a
 * device failure shows as NaN in obs and as KPM_ETIMEDOUT from
 * kpm_sync_status and rmft_iterate, rather than as a hang. */
int kpm_observables(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts,
                    const double* fields, const double* ab, double* obs,
                    double* omega, void* stream);

/* Up to n_iter self-consistency iterations of App. A: fields from params,
 * bounds, one KPM pass, then the mixing update (readings R1, R2).  params
 * (26*N doubles) and mu_eff (1 double) are read and updated in place; they may
 * be device pointers or host pointers (host buffers are staged through the
 * stream, copies included in the call).  phi: device or host, 4*N.
 * Blocks until the iterations are done (the host reads the residual after
 * each iteration).  Returns KPM_ENONFINITE on NaN/Inf. */
int rmft_iterate(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts,
                 const kpm_rmft_opts* ropts, const double* phi, double* params,
                 double* mu_eff, int n_iter, kpm_rmft_stats* stats, void* stream);

/* The two halves of one rmft_iterate iteration, for drivers that shard the
 * KPM pass over GPUs by sites (kpm_opts.site_begin/site_end) and merge the
 * observables themselves (App. A self-consistency; App. B: the start vectors
 * are independent).  rmft_prepare: fields from params at mu_eff with the mean
 * site energy taken out (reading R2), then the Gershgorin bounds (b = 0 exactly
 * with KPM_FLAG_PH_HALF in opts).  fields: 26 N, ab: 2 doubles, mu_out: 1
 * double (the Lagrange multiplier mu = mu_eff + <dW/dn|_{mu=0}>), all device;
 * phi, params, mu_eff device.  rmft_update: the mixing update of
 * rmft_iterate from the observables of the whole lattice (linear mixing;
 * anderson must be 0): params and mu_eff updated in place, obs overwritten by
 * the processed observables, stats_out (device, 2 doubles) = {max |p_new - p|,
 * <n_new> - n_target}.  Every rank that runs rmft_update on the same merged
 * obs computes bit-identical params. */
int rmft_prepare(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const double* phi,
                 const double* params, const double* mu_eff, double* fields, double* ab, double* mu_out,
                 void* stream);
int rmft_update(kpm_ctx* ctx, const kpm_model* model, const kpm_rmft_opts* ropts, double* params, double* obs,
                double* mu_eff, double* stats_out, void* stream);

/* Autotuner of the recursion launch: times two short passes (M = 18 and 34)
 * for every slab width in {D, 8192, ..., 128} (narrow slabs keep both
 * recursion vectors in L2), every column chunk that fits shared memory and
 * (FP32) one or two steps per launch, and for one step per launch the
 * three best band heights of a wave model of the launch (CTAs of
 * ceil(ny / bands) rows, one per SM; the first is the default of band_rows
 * = 0) and one band per column chunk, predicts the pass at opts->M from the
 * line through both times (per-slab start and gather plus M - 1 steps), and
 * writes the fastest (block_width, cols_per_block, band_rows,
 * KPM_FLAG_DOUBLE_STEP bit of flags) into *best (other fields copied from
 * *opts).  Results are cached per
 * (nx, ny, precision, KPM_FLAG_PH_HALF, probe_p, M) in the context (a cached
 * answer returns *best_ms_per_step = -1).  fields, ab: device, as for
 * kpm_observables.  best_ms_per_step: host double or NULL, the chosen
 * configuration's time per moment of the whole pass (all slabs), in ms. */
int kpm_autotune(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const double* fields,
                 const double* ab, kpm_opts* best, double* best_ms_per_step, void* stream);

/* Batched self-consistency (cells of uneven size, doping and field): up to
 * n_iter iterations of rmft_iterate's loop for ncell independent cells,
 * replayed as one CUDA graph per iteration.  FP32: every cell whose band of
 * ceil(ny / 8) lattice rows fits shared memory (nx up to 64 at ny = 32) runs
 * the persistent recursion: one launch per iteration for all of them, in
 * which a cluster of 8 CTAs holds a 16-column chunk of one cell on chip for
 * all M moments (work items longest first); cells that do not fit share one
 * batched step launch per Chebyshev step per shape, on concurrent streams.
 * FP64 runs the cells of a shape in sequence.  models, ropts, phis, params,
 * stats: arrays of ncell entries (host arrays; phis[c] and params[c] device
 * pointers of 4N_c and 26N_c doubles, updated in place); mu_eff: device array
 * of ncell doubles (updated); opts shared (M, precision; no site range).  At
 * most 64 cells of one shape in FP32; ropts[c].anderson must be 0 and
 * sync_every <= 1.  Stops early when every cell meets its tol; stats[c] as in
 * rmft_iterate, with recursion_ms the device time of the persistent launch
 * summed over the iterations (the same for every cell; 0 when no cell runs
 * it), recursion_bytes the cell's streaming-equivalent bytes of those
 * iterations (24 B per row-column and step) and recursion_launches 1. */
int rmft_iterate_batched(kpm_ctx* ctx, int ncell, const kpm_model* models, const kpm_opts* opts,
                         const kpm_rmft_opts* ropts, const double* const* phis, double* const* params,
                         double* mu_eff, int n_iter, kpm_rmft_stats* stats, void* stream);

/* Reverse-mode gradient of one KPM pass (App. B, Eqs. dFdH, dalphadH): for a
 * loss L with upstream gradients grad_obs = dL/d(obs) (26*N, the observable
 * layout; complex entries hold (dL/dRe, dL/dIm)) and grad_omega = dL/dOmega,
 * writes grad_fields = dL/d(eps, T, D) (26*N, field layout, same complex
 * convention) and, when grad_phi is not NULL, grad_phi = dL/dphi (4*N)
 * through the fields' dependence on the Peierls phases at order parameters
 * `params` (then phi and params are required).  The rescaling ab is held
 * fixed.  Backward recursion lambda_m = c_m + 2 h~ lambda_{m+1} -
 * lambda_{m+2} over all D unit columns (or those of the site range), with
 * the forward vectors alpha_m either
 *   ckpt_every >= 0: checkpointed every ckpt_every moments (0 = round(sqrt(M)))
 *     and recomputed per segment; scratch (2 ceil((M-1)/s) + s + 2) slab
 *     vectors within the context budget; or
 *   ckpt_every = KPM_REGENERATE: regenerated in descending m by the same
 *     recursion run backwards, alpha_{m-1} = 2 h~ alpha_m - alpha_{m+1}, from
 *     the last two vectors; these come from a forward sweep, or without one
 *     from the tail the last kpm_observables with KPM_FLAG_KEEP_TAIL left
 *     when its model, pass options, fields and ab equal this call's (checked
 *     on the device; one stream synchronisation); scratch 4 slab vectors.
 *     The recursion's rounding in reverse is bounded like its forward
 *     rounding (both run the neutrally stable three-term recurrence on
 *     eigenvalues in [-1, 1]).
 * Stencil-entry sums in FP64.  All pointers device. */
int kpm_backward(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const double* fields,
                 const double* ab, const double* grad_obs, double grad_omega, double* grad_fields,
                 const double* phi, const double* params, double* grad_phi, int ckpt_every, void* stream);

/* The same KPM pass as kpm_observables, for callers that cannot allocate
 * device memory: code running under a memory manager that owns the whole
 * device heap (a pre-sized arena that forbids other allocations) and code on
 * a latency-critical path where cudaMalloc/cudaFree would synchronise the
 * device.  The paper has no counterpart; this is an interface of this
 * library only.
 *
 * No context and no allocation: every intermediate lives in a file-scope
 * device array of 48 MiB (per GPU, held by every GPU that loads the library
 * until the process exits).  Calls outside stream capture resolve that
 * array's address with the device current (so a device reset that reloads the
 * module is followed); a call on a capturing stream reuses the address of the
 * last call outside capture on that device, so make one call before
 * capturing.  All calls on a device share the array: calls whose GPU work
 * overlaps (other streams, other host threads) race, so serialise them.  Each
 * call rewrites every scratch byte it reads.  The recursion slab is narrowed
 * to what fits (block_width is an upper bound); a lattice or M whose fixed
 * intermediates (4M doubles, 26N stencil entries, 10 accumulators per column,
 * one column chunk of both slabs) exceed 48 MiB returns KPM_EINVAL.
 * Arguments as for kpm_observables (all sites: site_begin = site_end = 0;
 * negative block_width or cols_per_block: KPM_EINVAL), device pointers of the
 * current device; result within rounding of kpm_observables (identical
 * arithmetic, possibly a different slab width).  The FP32 recursion's bounded
 * waits behave as in kpm_observables: a device failure shows as NaN in obs,
 * and kpm_sync_status (with any context of the device) reports and clears the
 * fault word. */
int kpm_observables_noalloc(const kpm_model* model, const kpm_opts* opts, const double* fields,
                            const double* ab, double* obs, double* omega, void* stream);

/* Vortex-profile order parameters (Sec. III, Eqs. giDelta and gm):
 *   Delta_i = 1/8 sum_{sigma, tau = +-x, +-y} g^t_i,sigma g^t_{i+tau},sigma (-1)^{tau_y}
 *             Delta_{i,i+tau,sigma} e^{i phi_{i,i+tau}},
 *   Delta_{ij,up} = F_ij, Delta_{ij,dn} = F_ji, the bond phase sign chosen so that
 *   Delta_i transforms like a pair at site i under gauge changes;
 *   M_i = (-1)^{x+y} g^{s,xy}_i / 4 sum_tau sqrt(g^{s,z}_{i,i+tau} / g^{s,xy}_{i,i+tau}) m_i.
 * phi (4N), params (26N): device.  delta_out: device, 2N doubles (re, im per
 * site); mag_out: device, N doubles. */
int kpm_order_parameters(kpm_ctx* ctx, const kpm_model* model, const double* phi, const double* params,
                         double* delta_out, double* mag_out, void* stream);

/* Local density of states (App. C, Eqs. N_i and Gij):
 *   N_i,up(w) = -(g^t_i,up)^2 Im G_(i,up)(w + i Gamma) / pi,
 *   N_i,dn(w) = -(g^t_i,dn)^2 Im G_(i,dn)(-w + i Gamma) / pi,
 *   Gamma = gamma_alpha |w| + gamma0   (the paper: 0.25 |w| + 3e-4),
 * with G_II(z) = [(z - h)^-1]_II evaluated as the Chebyshev series of the
 * resolvent truncated at opts->M terms: (1/a)(1/s) sum_m (2 - delta_m0) w^m
 * [T_m(h~)]_II, z~ = (z - b)/a, s = sqrt(z~^2 - 1), w = z~ - s, |w| < 1.  The
 * series converges like |w|^M, i.e. it needs M well above a / Gamma near the
 * spectrum.  The diagonal moments come from one recursion pass (all unit
 * vectors, or their probing estimate when opts->probe_p > 0); the sum over
 * m is one FP64 GEMM per spin (cuBLAS).  params: device, 26 N, for the
 * Gutzwiller weights (g^t_i,sigma)^2 (reading L1), or NULL for weights 1.
 * omega: host or device array of n_omega frequencies (units of t, energy 0 =
 * the chemical potential inside h).  ldos: device, [2][n_omega][N] (spin up,
 * spin down).  Scratch: M x 2N + 2 n_omega M doubles.  Not with
 * KPM_FLAG_PH_HALF (KPM_EINVAL); gamma0 must be > 0. */
int kpm_ldos(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const double* fields, const double* ab,
             const double* params, int n_omega, const double* omega, double gamma_alpha, double gamma0, double* ldos,
             void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KPM_H */
