// Internal declarations shared by the translation units of libkpm.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/kpm.h"

namespace kpm {

constexpr int kSlots = 10;     // accumulated entries per unit column (9 local rows + Omega)
constexpr int kCoef = 26;      // complex 2h~ entries per site (both Nambu rows, padded)
constexpr int kRedBlock = 256; // threads of the reduction kernels

// Launch geometry of the recursion kernel (shared with the host planner).
struct ChebPlan {
  int nx, ny;
  int64_t D;       // 2 N
  int64_t ldv;     // slab width padded to a multiple of cb (complex elements per row)
  int cb;          // columns per CTA
  int ylen;        // lattice rows marched per CTA
  int nthreads;
  size_t smem;     // dynamic shared memory per CTA
  int tma_rows;    // FP32 step: Nambu rows per TMA box of a window row (0: cp.async staging)
  // FP32 double-step kernel (two recursion steps per launch); cb2 = 0: not used
  int cb2;         // columns per CTA (divides cb)
  int ylen2;       // lattice rows per band
  size_t smem2;
  // slab column c holds unit vector J = (s0 + c) << js (js = 1: particle-hole
  // half pass over the columns (j, up) only; the pass covers D >> js columns)
  int js;
  // probing (probe_p > 0): slab column c holds the probing vector of colour
  // s0 + c (R = 2 probe_p^2 colours, phases from probe_seed)
  int probe_p;
  uint32_t probe_seed;
  const double2* xi;  // device table conj(xi_J) of the pass (probing only)
  double* rec;        // diagonal moments [T_m(h~)]_JJ, rec[m D + (J & 1) N + (J >> 1)] (or null)
};

// What slab column c of a launch holds (built from the plan and the slab offset).
struct ColMap {
  int64_t s0;
  int js;
  int probe_p;
  uint32_t seed;
  const double2* xi;  // conj(xi_J), J < D (probing)
  double* rec;        // diagonal-moment record (or null)
};
inline ColMap colmap(const ChebPlan& p, int64_t s0) { return ColMap{s0, p.js, p.probe_p, p.probe_seed, p.xi, p.rec}; }
// unit start vectors (D >> js) or probing vectors (2 p^2) of a pass
inline int64_t pass_columns(const ChebPlan& p) {
  return p.probe_p > 0 ? 2 * (int64_t)p.probe_p * p.probe_p : (p.D >> p.js);
}

// Per-cell pointers of a batch of equally shaped cells (FP32 recursion).
constexpr int kMaxBatch = 64;
struct BatchPtrs {
  void* A[kMaxBatch];
  void* B[kMaxBatch];
  const void* table[kMaxBatch];
  double2* acc[kMaxBatch];
  const double* am[kMaxBatch];
  const double* ao[kMaxBatch];
};

// ---------------------------------------------------------------- rmft_kernels.cu
cudaError_t launch_peierls(const kpm_model& m, double* phi, cudaStream_t s);
// fields = dW/d(params) at chemical potential mu; wsite (N doubles) = per-site W parts
cudaError_t launch_fields(const kpm_model& m, const double* phi, const double* params,
                          double mu, double* fields, double* wsite, cudaStream_t s);
// eps -= (mean(eps) + *mu_eff)   (mean over 2N site energies); mu_out = mu_eff + mean
cudaError_t launch_shift_eps(int N, double* fields, const double* mu_eff, double* mean_scratch,
                             double* mu_out, double* red, cudaStream_t s);
// symmetric: particle-hole symmetric spectrum, b = 0 and a = (1 + margin) max(hi, -lo)
cudaError_t launch_gershgorin(const kpm_model& m, const double* fields, double margin, double* ab,
                              double* red, cudaStream_t s, int symmetric = 0);
// out2 = {max deviation from eps_up = eps_dn, T_up = T_dn, D_ij = D_ji; max field modulus}
cudaError_t launch_ph_asym(const kpm_model& m, const double* fields, double* out2, double* red, cudaStream_t s);
// a_m (occupation) and a^Omega_m (grand potential) coefficients from device (a, b) at
// temperature T (0: closed-form step); half: a^Omega_m (1 + (-1)^m)
cudaError_t launch_coefficients(int M, const double* ab, double* am, double* ao, cudaStream_t s, int half = 0,
                                double temperature = 0.0);
// per-site table of 2h~ entries in precision T (kCoef complex per site)
cudaError_t launch_scale_table_f32(const kpm_model& m, const double* fields, const double* ab,
                                   float2* table, cudaStream_t s);
// double-float table: entries as float4 (re_hi, re_lo, im_hi, im_lo)
cudaError_t launch_scale_table_df(const kpm_model& m, const double* fields, const double* ab, float4* table,
                                  cudaStream_t s);
cudaError_t launch_scale_table_f64(const kpm_model& m, const double* fields, const double* ab,
                                   double2* table, cudaStream_t s);
// obs from accumulators; omega = a * sum Re acc[J][9] (if omega != null)
// half: particle-hole half pass (only the columns (j, up) accumulated);
// sites outside [sb, se) (se < 0: N) get zeros and no Omega part
cudaError_t launch_assemble(int nx, int ny, const double2* acc, const double* ab, double* obs, double* omega,
                            double* red, cudaStream_t s, int half = 0, int sb = 0, int se = -1);
// sum of a device array into *out (deterministic two-stage reduction)
cudaError_t launch_sum(const double* x, int64_t n, double* out, double* red, cudaStream_t s);
// Anderson mixing state (device): history ring dX, dF (m x L), previous x and f,
// current f (L each), Gram partials, gamma; L = 26 N + 1
struct AndersonState {
  int m = 0;
  double *dX = nullptr, *dF = nullptr, *xprev = nullptr, *fprev = nullptr, *fcur = nullptr, *gpart = nullptr,
         *gamma = nullptr;
};
size_t anderson_doubles(int N, int m);
AndersonState anderson_state(int N, int m, double* base);
// RMFT mixing update; writes stats = {residual, density_error} and updates mu_eff
// (linear mixing, or Anderson mixing when an && an->m > 0); rec (optional, 16
// doubles, rec[6..8] zero at the start of a call): record of the iteration,
// snap = {a, b, mu, omega} of its pass; an iteration after one that met tol
// changes nothing
cudaError_t launch_update(int N, double* params, double* obs, double* mu_eff, const kpm_rmft_opts& o,
                          double* stats, double* red, cudaStream_t s, double* rec = nullptr,
                          const double* snap = nullptr, const AndersonState* an = nullptr);
int reduce_scratch_doubles(int64_t n);

// ---------------------------------------------------------------- cheb_kernels.cu
ChebPlan plan_cheb(int nx, int ny, int64_t ldv_cols, int precision, int cb_request, int band_rows = 0);
// up to maxn band heights (lattice rows per CTA) for chunks column chunks of
// an ny-row lattice, best first by a wave model of the one-step kernels
int band_rows_candidates(int ny, int64_t chunks, int* out, int maxn);
// bytes of the per-site 2h~ table (kCoef complex entries)
size_t table_bytes_per_site(int precision);
cudaError_t cheb_prepare(const ChebPlan& p, int precision);
// zero V0/acc slab, V0 = unit vectors of columns [s0, s0 + b), acc init with a_0 terms
cudaError_t launch_cheb_init(const ChebPlan& p, int precision, void* V0, int64_t s0,
                             double2* acc, const double* am, const double* ao, cudaStream_t s);
// one recursion step. mode 0: Vout = h~ Vcur (first step); mode 1: Vout = 2h~ Vcur - Vprev
// (Vprev = nullptr: in place, Vprev = Vout), accumulating a_m Vcur into acc unless acc is null
// (m = step index of Vcur)
cudaError_t launch_cheb_step(const ChebPlan& p, int precision, const void* table, const void* Vcur,
                             void* Vout, int64_t s0, double2* acc, const double* am,
                             const double* ao, int m, int mode, cudaStream_t s, const void* Vprev = nullptr);
// FP32 double step: Vout1 = V_{m+1}, Vout2 = V_{m+2} from Vprev = V_{m-1}, Vcur = V_m
// (four distinct slabs), accumulating a_m V_m and a_{m+1} V_{m+1} unless acc is null
cudaError_t launch_cheb_step2(const ChebPlan& p, const void* table, const void* Vprev, const void* Vcur,
                              void* Vout1, void* Vout2, int64_t s0, double2* acc, const double* am,
                              const double* ao, int m, cudaStream_t s);
// batched FP32 step over ncell cells of one shape (plan p, full-width slabs);
// with p.tma_rows > 0 and `maps` (device copy of the 2 ncell tensor maps that
// encode_batch_maps writes to host memory, batch_maps_bytes(ncell) bytes,
// 64-byte aligned) the TMA-staged kernel runs, else the cp.async one
cudaError_t cheb_prepare_batched(const ChebPlan& p);
size_t batch_maps_bytes(int ncell);
cudaError_t encode_batch_maps(const ChebPlan& p, int ncell, const BatchPtrs& b, void* host_maps);
cudaError_t launch_cheb_step_batched(const ChebPlan& p, int ncell, const BatchPtrs& b, int m, int mode,
                                     cudaStream_t s, const void* maps = nullptr);
// device fault word of the TMA-staged FP32 step (bit 0: a bounded wait
// expired; bit 1: shared memory misaligned for TMA); sticky for the process
cudaError_t read_step_fault(unsigned int* out);
cudaError_t clear_step_fault();
// failure-path test hook: the next drop_copies CTAs of the TMA step skip one
// window copy; bounded-wait limit of later launches (0: the default 2 s)
cudaError_t set_step_failure_test(int drop_copies, uint64_t wait_limit_ns);
// table conj(xi_J) of the probing phases, J < D
cudaError_t launch_probe_phases(const ChebPlan& p, double2* xi_conj, cudaStream_t s);
// acc += a_m V[local rows] for the slab's columns (no recursion)
cudaError_t launch_cheb_gather(const ChebPlan& p, int precision, const void* V, int64_t s0,
                               double2* acc, const double* am, const double* ao, int m,
                               cudaStream_t s);

// persistent batched FP32 recursion: clusters of kPClu CTAs, one item = one
// chunk of persist_columns() unit columns of one cell for all M moments
// (moment sums written to cell.acc, including the a_0 terms and the last moment)
constexpr int kPClu = 8;
struct PCell {
  int nx, ny;
  const float2* table;  // the cell's 2h~ table (FP32)
  double2* acc;         // its moment sums [D][kSlots]
  const double* am;
  const double* ao;
};
struct PItem {
  int cell;  // index into the cell array
  int q0;    // first unit column of the chunk
};
size_t persist_smem_bytes(int nx, int ny);
int persist_columns();
// sets the kernel's shared-memory limit; *max_clusters = co-resident clusters at `smem`
cudaError_t persist_prepare(size_t smem, int* max_clusters);
// device bytes of the boundary-row exchange buffer of nclusters clusters
size_t persist_exchange_bytes(int nclusters, int nx_max);
// items are taken from *counter (zero before the launch) in list order; xbuf:
// persist_exchange_bytes(nclusters, nx_max) device bytes, nx_max >= every cell's nx
cudaError_t launch_cheb_persist(const PCell* cells, const PItem* items, int nitems, int* counter, int M, int nclusters,
                                size_t smem, void* xbuf, int nx_max, cudaStream_t s);

// ---------------------------------------------------------------- kpm_adjoint.cu
// *same = 1 when a = b (n doubles) and c = d (k doubles) bit for bit; flag: a
// device int, host: a pinned host int; synchronises s
cudaError_t launch_same_doubles(const double* a, const double* b, int64_t n, const double* c, const double* d, int k,
                                int* flag, int* host, int* same, cudaStream_t s);
// seed weights w[J][10] of every unit column from the upstream gradients (zero
// for the columns of sites outside [sb, se), se < 0: N)
cudaError_t launch_seed_weights(int nx, int ny, const double* grad_obs, const double* ab, double g_omega,
                                double2* w, cudaStream_t s, int sb = 0, int se = -1);
// lambda[K_s(J), c] += coef_s(m) w[J][s] over the slab's columns
cudaError_t launch_seed_scatter(const ChebPlan& p, int prec, void* lam, int64_t s0, const double2* w,
                                const double* am, const double* ao, int m, cudaStream_t s);
// column sets of the stencil-entry sums (partial buffer P holds grad_groups x D x 13 entries)
int grad_groups(const ChebPlan& p, int prec);
// P[set][I][k] += coef sum_{c in set} lam[I, c] conj(alpha[K_k(I), c]) over the 13 stencil entries of each row
cudaError_t launch_grad_accum(const ChebPlan& p, int prec, const void* lam, const void* alpha, double coef,
                              double2* P, cudaStream_t s);
// G[I][k] = sum over the sets of P[set][I][k] (fixed order)
cudaError_t launch_grad_reduce(int64_t D, int groups, const double2* P, double2* G, cudaStream_t s);
// dL/d(eps, T, D) from G (gradient in h~) with h~ = (h - b)/a
cudaError_t launch_grad_fields(int nx, int ny, const double2* G, const double* ab, double* out, cudaStream_t s);
// dL/dphi through the fields' dependence on the Peierls phases (rmft_kernels.cu)
cudaError_t launch_phi_grad(const kpm_model& m, const double* phi, const double* params, const double* grad_fields,
                            double* grad_phi, cudaStream_t s);

// ---------------------------------------------------------------- kpm_peaks.cu
// FMA throughput of the FP64 and FP32 pipes: out = {FP64 TFLOP/s, FP32 TFLOP/s,
// packed f32x2 TFLOP/s, median SM MHz}; scratch: peak_scratch_bytes(sms) device bytes
size_t peak_scratch_bytes(int sms);
cudaError_t measure_alu_peaks(int sms, void* scratch, double* out, cudaStream_t s);

// ---------------------------------------------------------------- kpm_ldos.cu
// C[sigma][k][m] of the resolvent series (see kpm_ldos.cu)
cudaError_t launch_ldos_coefficients(int M, int nw, const double* omega, double alpha, double gamma0,
                                     const double* ab, double* C, cudaStream_t s);
// ldos = -w/pi * (moments x coefficients), one FP64 GEMM per spin; null or an error message
const char* ldos_contract(void* cublas, int M, int nw, int64_t N, const double* C, const double* rec, double* ldos,
                          const double* wgt, cudaStream_t s);
void* cublas_create();
void cublas_destroy(void* h);
// physical pairing Delta_i (2N: re, im) and staggered magnetisation M_i (N) (rmft_kernels.cu)
cudaError_t launch_order_parameters(const kpm_model& m, const double* phi, const double* params, double* delta_out,
                                    double* mag_out, cudaStream_t s);
// (g^t_{i sigma})^2 per site and spin, [2][N] (rmft_kernels.cu)
cudaError_t launch_gt_weights(const kpm_model& m, const double* params, double* w, cudaStream_t s);

}  // namespace kpm
