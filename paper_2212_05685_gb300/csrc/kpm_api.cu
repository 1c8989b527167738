// C ABI of libkpm.so: context and scratch management, argument checks, the
// ordering of one KPM pass (coefficients, rescaled stencil table, slab
// recursions, assembly) and of one self-consistency iteration, captured once
// into a CUDA graph and replayed.
#include <cuda.h>
#include <math.h>
#include <string.h>

#include <new>

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "kpm_internal.cuh"

using namespace kpm;

struct kpm_ctx {
  int device = 0;
  cudaStream_t cap = nullptr;  // capture stream of the iteration graph
  std::string err;
  uint64_t budget = 24ull << 30;

  // scratch (owned)
  void* slab[4] = {nullptr, nullptr, nullptr, nullptr};  // two, or four for the double-step recursion
  int slab_n = 0;
  size_t slab_bytes = 0;
  double2* xi = nullptr;  // probing phases conj(xi_J) of the current pass
  size_t xi_bytes = 0;
  // LDOS: diagonal-moment record, coefficient matrix, weights, frequencies, cuBLAS handle
  double* ldos_buf = nullptr;
  size_t ldos_buf_bytes = 0;
  void* cublas = nullptr;
  double2* acc = nullptr;
  size_t acc_bytes = 0;
  void* table = nullptr;
  size_t table_bytes = 0;
  double* am = nullptr;
  double* ao = nullptr;
  size_t coef_n = 0;
  double* red = nullptr;        // reduction partials
  double* fields = nullptr;     // 26 N
  double* obs = nullptr;        // 26 N
  double* wsite = nullptr;      // N
  double* dparams = nullptr;    // 26 N (host-pointer staging)
  double* dphi = nullptr;       // 4 N
  size_t site_n = 0;
  double* misc = nullptr;       // [0..1] ab, [2] mu, [3] omega, [4..5] stats, [6] mean, [7] mu_eff, [8] W,
                                // [16..31] record of the iteration loop (launch_update)
  double* and_buf = nullptr;    // Anderson mixing state
  size_t and_bytes = 0;
  double* peak_buf = nullptr;   // scratch of kpm_measure_peaks
  size_t peak_bytes = 0;
  // tail of the last kpm_observables with KPM_FLAG_KEEP_TAIL: per slab the last
  // two recursion vectors (alpha_{M-2}, alpha_{M-1}); the fields and ab it ran
  // on (26 N + 2 doubles) and the pass it belongs to
  void* tail = nullptr;
  size_t tail_bytes = 0;
  double* tail_in = nullptr;
  size_t tail_in_bytes = 0;
  bool tail_valid = false;
  kpm_model tail_model;
  kpm_opts tail_opts;
  int64_t tail_width = 0, tail_c0 = 0, tail_c1 = 0;
  // adjoint scratch: checkpoints, segment, lambda buffers; stencil gradient; seed weights
  void* bwd = nullptr;
  size_t bwd_bytes = 0;
  double2* Gacc = nullptr;
  size_t Gacc_bytes = 0;
  double2* wseed = nullptr;
  size_t wseed_bytes = 0;
  double* host_misc = nullptr;  // pinned mirror of misc

  // events around the recursion steps of the captured iteration
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int launches = 0;      // kernels per captured iteration
  int rec_launches = 0;  // recursion-step kernels per captured iteration
  double rec_bytes = 0;  // their algorithmic bytes

  // batched iteration: per-cell scratch, fork streams, cached graph
  struct Cell {
    void* mem = nullptr;  // one allocation per cell
    size_t bytes = 0;
    double *fields, *obs, *am, *ao, *misc;
    double2* acc;
    void *table, *A, *B;
    int cls;
  };
  std::vector<Cell> cells;
  std::vector<cudaStream_t> fork;
  std::vector<cudaEvent_t> fork_ev;
  cudaEvent_t join_ev = nullptr;
  double* bred = nullptr;          // reduction partials (cells run in sequence on one stream)
  double* bhost = nullptr;         // pinned mirror of the cells' misc blocks
  size_t bhost_n = 0;
  cudaGraphExec_t bgraph = nullptr;
  std::vector<char> bkey;
  std::vector<void*> bmaps;        // per shape class: device copy of its cells' slab tensor maps
  // persistent recursion of the batch: cell table, work items (longest first),
  // item counter; events around its launch
  void* pbuf = nullptr;
  size_t pbuf_bytes = 0;
  cudaEvent_t pev[2] = {nullptr, nullptr};
  int p_launched = 0;              // 1 when the captured batch graph holds the persistent launch
  double p_bytes = 0;              // its streaming-equivalent bytes per iteration

  // autotuned (block_width, cols_per_block, double-step flag, band_rows) per (nx, ny, precision, half pass,
  // probe_p, M)
  std::map<std::tuple<int, int, int, int, int, int>, std::tuple<int, int, int, int>> tuned;

  // cached iteration graph
  cudaGraphExec_t graph = nullptr;
  struct Key {
    kpm_model m;
    kpm_opts o;
    kpm_rmft_opts r;
    const double* phi;
    double* params;
    double* mu_eff;
  } key;
  bool key_valid = false;
};

namespace {

int fail(kpm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(kpm_ctx* c, cudaError_t e, const char* where) {
  cudaGetLastError();  // clear a non-sticky error so later launch checks see their own status
  return fail(c, KPM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define KPM_CU(expr)                                  \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_model(kpm_ctx* ctx, const kpm_model* m) {
  if (!m) return fail(ctx, KPM_EINVAL, "model is null");
  if (m->nx < 2 || m->ny < 2) return fail(ctx, KPM_EINVAL, "lattice needs nx, ny >= 2");
  if ((int64_t)m->nx * m->ny > (1 << 26)) return fail(ctx, KPM_EINVAL, "lattice too large");
  return KPM_OK;
}

int check_dev(kpm_ctx* ctx, const void* p, const char* name) {
  if (!p) return fail(ctx, KPM_EINVAL, std::string(name) + " is null");
  if (((uintptr_t)p) % 8) return fail(ctx, KPM_EINVAL, std::string(name) + " is not 8-byte aligned");
  if (!is_device_ptr(p)) return fail(ctx, KPM_EINVAL, std::string(name) + " is not a device pointer");
  return KPM_OK;
}

template <typename T>
int ensure(kpm_ctx* ctx, T** p, size_t* have, size_t need_bytes) {
  if (*p && *have >= need_bytes) return KPM_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc((void**)p, need_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, KPM_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  *have = need_bytes;
  return KPM_OK;
}

void drop_graph(kpm_ctx* ctx) {
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  ctx->graph = nullptr;
  ctx->key_valid = false;
}

int ensure_site_scratch(kpm_ctx* ctx, int N) {
  if (ctx->site_n >= (size_t)N && ctx->fields) return KPM_OK;
  drop_graph(ctx);
  double** bufs[5] = {&ctx->fields, &ctx->obs, &ctx->wsite, &ctx->dparams, &ctx->dphi};
  const size_t sizes[5] = {26, 26, 1, 26, 4};
  for (int k = 0; k < 5; ++k) {
    if (*bufs[k]) cudaFree(*bufs[k]);
    *bufs[k] = nullptr;
    if (cudaMalloc((void**)bufs[k], sizes[k] * (size_t)N * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      ctx->site_n = 0;
      return fail(ctx, KPM_ENOMEM, "cudaMalloc of per-site scratch failed");
    }
  }
  ctx->site_n = N;
  return KPM_OK;
}

struct PassPlan {
  ChebPlan cheb;
  int64_t width;  // unit columns per slab
  size_t elem;    // bytes per complex
  bool dbl;       // FP32 double-step recursion (four slabs)
  int64_t c0, c1; // pass columns [c0, c1) (all: 0, pass_columns)
  int sb, se;     // sites whose observables the pass writes (all: 0, N)
  bool ranged;    // a proper sub-range of the sites
};

// the widest equal split of D unit columns into slabs of at most `width`
// columns (a ragged last slab would cost a full slab's launches)
int64_t balanced_width(int64_t D, int64_t width) {
  if (width >= D) return D;
  const int64_t n = (D + width - 1) / width;
  return (D + n - 1) / n;
}

int plan_pass(kpm_ctx* ctx, const kpm_model* m, const kpm_opts* o, PassPlan* pp) {
  if (!o) return fail(ctx, KPM_EINVAL, "opts is null");
  if (o->M < 1) return fail(ctx, KPM_EINVAL, "M must be >= 1");
  if (o->precision != KPM_FP32 && o->precision != KPM_FP64 && o->precision != KPM_DF64)
    return fail(ctx, KPM_EINVAL, "unknown precision");
  if (o->block_width < 0 || o->cols_per_block < 0) return fail(ctx, KPM_EINVAL, "negative block width");
  if (o->band_rows < 0) return fail(ctx, KPM_EINVAL, "negative band_rows");
  const int64_t D = 2 * (int64_t)m->nx * m->ny;
  pp->elem = o->precision == KPM_FP32 ? 8 : 16;
  if (!(o->temperature >= 0.0 && o->temperature < 1e300)) return fail(ctx, KPM_EINVAL, "temperature must be finite and >= 0");
  const int pp_ = o->probe_p;
  if (pp_ < 0 || pp_ == 1 || (pp_ > 0 && (m->nx % pp_ != 0 || m->ny % pp_ != 0)))
    return fail(ctx, KPM_EINVAL, "probe_p must be 0 or >= 2 and divide nx and ny");
  if (pp_ > 0 && (o->flags & KPM_FLAG_PH_HALF))
    return fail(ctx, KPM_EINVAL, "probing and KPM_FLAG_PH_HALF do not combine");
  const int N = m->nx * m->ny;
  pp->sb = 0;
  pp->se = N;
  pp->ranged = false;
  if (o->site_begin != 0 || o->site_end != 0) {
    if (!(o->site_begin >= 0 && o->site_begin < o->site_end && o->site_end <= N))
      return fail(ctx, KPM_EINVAL, "site range must satisfy 0 <= site_begin < site_end <= N");
    pp->sb = o->site_begin;
    pp->se = o->site_end;
    pp->ranged = !(pp->sb == 0 && pp->se == N);
    if (pp->ranged && pp_ > 0) return fail(ctx, KPM_EINVAL, "probing and a site range do not combine");
    if (pp->ranged && (o->flags & KPM_FLAG_PH_HALF))
      return fail(ctx, KPM_EINVAL, "KPM_FLAG_PH_HALF and a site range do not combine");
  }
  const bool want_dbl = o->precision == KPM_FP32 && (o->flags & KPM_FLAG_DOUBLE_STEP) && pp_ == 0;
  const int js = (o->flags & KPM_FLAG_PH_HALF) ? 1 : 0;
  // start vectors of the pass: unit columns (those of the site range), or R = 2 p^2 probing vectors
  pp->c0 = pp->ranged ? 2 * (int64_t)pp->sb : 0;
  pp->c1 = pp->ranged ? 2 * (int64_t)pp->se : (pp_ > 0 ? std::min<int64_t>(D, 2 * (int64_t)pp_ * pp_) : (D >> js));
  const int64_t ncols = pp->c1 - pp->c0;
  int64_t width = o->block_width > 0 ? std::min<int64_t>(o->block_width, ncols) : ncols;
  if (o->block_width == 0) {
    const int64_t fit = (int64_t)(ctx->budget / ((want_dbl ? 4 : 2) * (uint64_t)D * pp->elem));
    width = balanced_width(ncols, std::min<int64_t>(width, std::max<int64_t>(fit, 1)));
  }
  pp->cheb = plan_cheb(m->nx, m->ny, width, o->precision, o->cols_per_block, o->band_rows);
  pp->cheb.js = js;
  pp->cheb.probe_p = pp_;
  pp->cheb.probe_seed = (uint32_t)o->probe_seed;
  if (pp->cheb.cb == 0) return fail(ctx, KPM_EINVAL, "lattice row too wide for the shared-memory window");
  // slabs advance by the padded width: every unit column belongs to exactly one slab
  pp->width = pp->cheb.ldv;
  pp->dbl = want_dbl && pp->cheb.cb2 > 0;
  return KPM_OK;
}

int ensure_pass_scratch(kpm_ctx* ctx, const kpm_model* m, const kpm_opts* o, const PassPlan& pp) {
  const int64_t D = pp.cheb.D;
  const size_t slab = (size_t)D * pp.cheb.ldv * pp.elem;
  const int nslab = pp.dbl ? 4 : 2;
  int r;
  if (ctx->slab_bytes < slab || ctx->slab_n < nslab) {
    drop_graph(ctx);
    for (int k = 0; k < 4; ++k) {
      if (ctx->slab[k]) cudaFree(ctx->slab[k]);
      ctx->slab[k] = nullptr;
    }
    ctx->slab_bytes = 0;
    ctx->slab_n = 0;
    for (int k = 0; k < nslab; ++k) {
      if (cudaMalloc(&ctx->slab[k], slab) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, KPM_ENOMEM, "cudaMalloc of the recursion slabs failed");
      }
    }
    ctx->slab_bytes = slab;
    ctx->slab_n = nslab;
  }
  const size_t accb = (size_t)D * kSlots * sizeof(double2);
  if (ctx->acc_bytes < accb) drop_graph(ctx);
  if ((r = ensure(ctx, &ctx->acc, &ctx->acc_bytes, accb))) return r;
  if (pp.cheb.probe_p > 0) {
    if (ctx->xi_bytes < (size_t)D * sizeof(double2)) drop_graph(ctx);
    if ((r = ensure(ctx, &ctx->xi, &ctx->xi_bytes, (size_t)D * sizeof(double2)))) return r;
  }
  const size_t tb = (size_t)m->nx * m->ny * table_bytes_per_site(o->precision);
  if (ctx->table_bytes < tb) drop_graph(ctx);
  if ((r = ensure(ctx, &ctx->table, &ctx->table_bytes, tb))) return r;
  if (ctx->coef_n < (size_t)o->M) {
    drop_graph(ctx);
    if (ctx->am) cudaFree(ctx->am);
    if (ctx->ao) cudaFree(ctx->ao);
    ctx->am = ctx->ao = nullptr;
    ctx->coef_n = 0;
    if (cudaMalloc(&ctx->am, o->M * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctx->ao, o->M * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, KPM_ENOMEM, "cudaMalloc of coefficients failed");
    }
    ctx->coef_n = o->M;
  }
  if (!ctx->red) {
    if (cudaMalloc(&ctx->red, reduce_scratch_doubles(0) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, KPM_ENOMEM, "cudaMalloc of reduction scratch failed");
    }
  }
  cudaError_t e = cheb_prepare(pp.cheb, o->precision);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cheb_prepare");
  return KPM_OK;
}

// enqueue one KPM pass: fields + ab (device) -> obs, omega
// When `events` is set, ctx->ev[0]/ev[1] are recorded on `s` around the
// recursion-step launches (first step of the first slab to the last step of
// the last slab); *launches / *rec_launches count the kernels enqueued.
int enqueue_pass(kpm_ctx* ctx, const kpm_model* m, const kpm_opts* o, const PassPlan& pp, const double* fields,
                 const double* ab, double* obs, double* omega, cudaStream_t s, bool events = false,
                 int* launches = nullptr, int* rec_launches = nullptr, double* rec_bytes = nullptr,
                 double* diag_record = nullptr, void* tail = nullptr) {
  ChebPlan p = pp.cheb;
  p.rec = diag_record;
  int nl0 = 0;
  if (p.probe_p > 0) {
    p.xi = ctx->xi;
    KPM_CU(launch_probe_phases(p, ctx->xi, s));
    nl0 = 1;
  }
  const int M = o->M;
  const int prec = o->precision;
  int nl = 0, nr = 0;
  double nb = 0.0;
  const double vec = (double)p.D * (double)p.ldv * (double)pp.elem;  // bytes of one slab vector
  KPM_CU(launch_coefficients(M, ab, ctx->am, ctx->ao, s, p.js, o->temperature));
  if (prec == KPM_FP32)
    KPM_CU(launch_scale_table_f32(*m, fields, ab, (float2*)ctx->table, s));
  else if (prec == KPM_DF64)
    KPM_CU(launch_scale_table_df(*m, fields, ab, (float4*)ctx->table, s));
  else
    KPM_CU(launch_scale_table_f64(*m, fields, ab, (double2*)ctx->table, s));
  nl += 2;
  for (int64_t s0 = pp.c0; s0 < pp.c1; s0 += pp.width) {
    // X0 = V_{mm-1}, X1 = V_mm; Y0, Y1 the free pair of the double-step recursion
    void* X0 = ctx->slab[0];
    void* X1 = ctx->slab[1];
    void* Y0 = pp.dbl ? ctx->slab[2] : nullptr;
    void* Y1 = pp.dbl ? ctx->slab[3] : nullptr;
    KPM_CU(launch_cheb_init(p, prec, X0, s0, ctx->acc, ctx->am, ctx->ao, s));
    nl += 1;
    if (events && s0 == pp.c0) KPM_CU(cudaEventRecordWithFlags(ctx->ev[0], s, cudaEventRecordExternal));
    if (M >= 2) {
      KPM_CU(launch_cheb_step(p, prec, ctx->table, X0, X1, s0, ctx->acc, ctx->am, ctx->ao, 0, 0, s));
      nr += 1;
      nb += 2 * vec;
    }
    int mm = 1;  // highest vector index computed so far
    if (pp.dbl) {
      for (; mm + 2 <= M - 1; mm += 2) {
        KPM_CU(launch_cheb_step2(p, ctx->table, X0, X1, Y0, Y1, s0, ctx->acc, ctx->am, ctx->ao, mm, s));
        nr += 1;
        nb += 4 * vec;
        std::swap(X0, Y0);
        std::swap(X1, Y1);
      }
    }
    for (; mm + 1 <= M - 1; ++mm) {
      // V_{mm+1} = 2 h~ V_mm - V_{mm-1} in place over V_{mm-1}
      KPM_CU(launch_cheb_step(p, prec, ctx->table, X1, X0, s0, ctx->acc, ctx->am, ctx->ao, mm, 1, s));
      nr += 1;
      nb += 3 * vec;
      std::swap(X0, X1);
    }
    if (events && s0 + pp.width >= pp.c1) KPM_CU(cudaEventRecordWithFlags(ctx->ev[1], s, cudaEventRecordExternal));
    if (M >= 2) {
      KPM_CU(launch_cheb_gather(p, prec, X1, s0, ctx->acc, ctx->am, ctx->ao, M - 1, s));
      nl += 1;
      if (tail) {  // alpha_{M-2}, alpha_{M-1} of this slab for a later backward pass
        char* t = static_cast<char*>(tail) + (size_t)(2 * ((s0 - pp.c0) / pp.width)) * (size_t)vec;
        KPM_CU(cudaMemcpyAsync(t, X0, (size_t)vec, cudaMemcpyDeviceToDevice, s));
        KPM_CU(cudaMemcpyAsync(t + (size_t)vec, X1, (size_t)vec, cudaMemcpyDeviceToDevice, s));
      }
    }
  }
  KPM_CU(launch_assemble(m->nx, m->ny, ctx->acc, ab, obs, omega, ctx->red, s, p.js, pp.sb, pp.se));
  nl += omega ? 2 : 1;
  if (launches) *launches = nl0 + nl + nr;
  if (rec_launches) *rec_launches = nr;
  if (rec_bytes) *rec_bytes = nb;
  return KPM_OK;
}

constexpr int kMisc = 32;  // doubles of ctx->misc / host_misc
constexpr int kRec = 16;   // offset of the iteration record in misc

int ensure_misc(kpm_ctx* ctx) {
  if (ctx->misc) return KPM_OK;
  if (cudaMalloc(&ctx->misc, kMisc * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KPM_ENOMEM, "cudaMalloc failed");
  }
  if (cudaMallocHost(&ctx->host_misc, kMisc * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KPM_ENOMEM, "cudaMallocHost failed");
  }
  cudaMemset(ctx->misc, 0, kMisc * sizeof(double));
  return KPM_OK;
}

// KPM_FLAG_PH_HALF precondition: fields in the particle-hole symmetric sector
// within 1e-12 of the largest field, and (ab given) |b| <= 1e-12 a.  Reads two
// device scalars back, so it synchronises the stream.
int check_ph_sector(kpm_ctx* ctx, const kpm_model* m, const double* fields, const double* ab, cudaStream_t s) {
  int r;
  if ((r = ensure_misc(ctx))) return r;
  KPM_CU(launch_ph_asym(*m, fields, ctx->misc + 10, ctx->red, s));
  KPM_CU(cudaMemcpyAsync(ctx->host_misc + 10, ctx->misc + 10, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (ab) KPM_CU(cudaMemcpyAsync(ctx->host_misc + 12, ab, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  KPM_CU(cudaStreamSynchronize(s));
  const double dev = ctx->host_misc[10], mag = ctx->host_misc[11];
  if (!(dev <= 1e-12 * std::max(1.0, mag)))
    return fail(ctx, KPM_EINVAL, "KPM_FLAG_PH_HALF: the fields are not particle-hole symmetric "
                                 "(need eps_up = eps_dn, T_up = T_dn, D_ij = D_ji)");
  if (ab && !(fabs(ctx->host_misc[13]) <= 1e-12 * ctx->host_misc[12]))
    return fail(ctx, KPM_EINVAL, "KPM_FLAG_PH_HALF: the rescaling centre b must be 0");
  return KPM_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool same_key(const kpm_ctx::Key& a, const kpm_ctx::Key& b) { return memcmp(&a, &b, sizeof(a)) == 0; }

}  // namespace

extern "C" {

const char* kpm_strerror(int status) {
  switch (status) {
    case KPM_OK: return "ok";
    case KPM_EINVAL: return "invalid argument";
    case KPM_ENOMEM: return "out of device memory";
    case KPM_ECUDA: return "CUDA error";
    case KPM_ENONFINITE: return "non-finite value in an output";
    case KPM_ETIMEDOUT: return "bounded device wait expired";
    case KPM_ENOTCONV: return "not converged";
    default: return "unknown status";
  }
}

const char* kpm_last_error(const kpm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int kpm_create(kpm_ctx** out, int device) {
  if (!out) return KPM_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return KPM_EINVAL;
  }
  kpm_ctx* ctx = new (std::nothrow) kpm_ctx();
  if (!ctx) return KPM_ENOMEM;
  ctx->device = device;
  DeviceGuard g(device);
  if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&ctx->ev[0]) != cudaSuccess || cudaEventCreate(&ctx->ev[1]) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    delete ctx;
    return KPM_ECUDA;
  }
  *out = ctx;
  return KPM_OK;
}

int kpm_destroy(kpm_ctx* ctx) {
  if (!ctx) return KPM_EINVAL;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  drop_graph(ctx);
  cublas_destroy(ctx->cublas);
  for (void* p : {ctx->slab[0], ctx->slab[1], ctx->slab[2], ctx->slab[3], (void*)ctx->xi, (void*)ctx->ldos_buf,
                  (void*)ctx->and_buf, (void*)ctx->peak_buf, ctx->tail, (void*)ctx->tail_in,
                  (void*)ctx->acc, ctx->table, (void*)ctx->am, (void*)ctx->ao,
                  (void*)ctx->red, (void*)ctx->fields, (void*)ctx->obs, (void*)ctx->wsite, (void*)ctx->dparams,
                  (void*)ctx->dphi, (void*)ctx->misc, ctx->bwd, (void*)ctx->Gacc, (void*)ctx->wseed})
    if (p) cudaFree(p);
  if (ctx->host_misc) cudaFreeHost(ctx->host_misc);
  if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
  for (auto& c : ctx->cells)
    if (c.mem) cudaFree(c.mem);
  for (void* p : ctx->bmaps) cudaFree(p);
  if (ctx->pbuf) cudaFree(ctx->pbuf);
  for (cudaEvent_t e : ctx->pev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t st : ctx->fork) cudaStreamDestroy(st);
  for (cudaEvent_t e : ctx->fork_ev) cudaEventDestroy(e);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  if (ctx->bred) cudaFree(ctx->bred);
  if (ctx->bhost) cudaFreeHost(ctx->bhost);
  for (cudaEvent_t e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  delete ctx;
  return KPM_OK;
}

// KPM_ETIMEDOUT / KPM_ECUDA for a fault recorded by the FP32 recursion, else
// 0; a recorded fault is cleared once the device is idle (the launches that
// saw it have written NaN by then)
static int device_fault_status(kpm_ctx* ctx) {
  unsigned int f = 0;
  cudaError_t e = read_step_fault(&f);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the device fault word");
  if (f == 0u) return KPM_OK;
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(ctx, e, "cudaDeviceSynchronize");
  if ((e = clear_step_fault()) != cudaSuccess) return cuda_fail(ctx, e, "clearing the device fault word");
  if (f & 1u)
    return fail(ctx, KPM_ETIMEDOUT,
                "a bounded wait of the FP32 recursion expired: the outputs of that launch, and of every FP32 "
                "recursion launch after it until this report, are NaN");
  return fail(ctx, KPM_ECUDA, "shared memory of the FP32 recursion was not aligned for TMA: outputs are NaN");
}

int kpm_sync_status(kpm_ctx* ctx, void* stream) {
  if (!ctx) return KPM_EINVAL;
  DeviceGuard g(ctx->device);
  KPM_CU(cudaStreamSynchronize((cudaStream_t)stream));
  return device_fault_status(ctx);
}

int kpm_inject_lost_copy(kpm_ctx* ctx, int count, double wait_limit_s) {
  if (!ctx) return KPM_EINVAL;
  if (count < 0 || !(wait_limit_s < 3600.0)) return fail(ctx, KPM_EINVAL, "count must be >= 0, wait limit < 1 h");
  DeviceGuard g(ctx->device);
  KPM_CU(cudaDeviceSynchronize());
  const uint64_t ns = wait_limit_s > 0.0 ? (uint64_t)(wait_limit_s * 1e9) : 0;
  KPM_CU(set_step_failure_test(count, ns < 1000 && wait_limit_s > 0.0 ? 1000 : ns));
  return KPM_OK;
}

int kpm_measure_peaks(kpm_ctx* ctx, double* out, void* stream) {
  if (!ctx || !out) return KPM_EINVAL;
  DeviceGuard g(ctx->device);
  int sms = 0;
  KPM_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  int r;
  if ((r = ensure(ctx, &ctx->peak_buf, &ctx->peak_bytes, peak_scratch_bytes(sms)))) return r;
  KPM_CU(measure_alu_peaks(sms, ctx->peak_buf, out, (cudaStream_t)stream));
  return KPM_OK;
}

int kpm_set_scratch_budget(kpm_ctx* ctx, uint64_t bytes) {
  if (!ctx || bytes < (1u << 20)) return KPM_EINVAL;
  ctx->budget = bytes;
  return KPM_OK;
}

int kpm_peierls_phases(kpm_ctx* ctx, const kpm_model* model, double* phi, void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if ((r = check_dev(ctx, phi, "phi"))) return r;
  DeviceGuard g(ctx->device);
  KPM_CU(launch_peierls(*model, phi, (cudaStream_t)stream));
  return KPM_OK;
}

int kpm_build_H(kpm_ctx* ctx, const kpm_model* model, const double* phi, const double* params, double mu,
                double* fields, double* w_out, void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if ((r = check_dev(ctx, phi, "phi")) || (r = check_dev(ctx, params, "params")) ||
      (r = check_dev(ctx, fields, "fields")))
    return r;
  if (w_out && (r = check_dev(ctx, w_out, "w_out"))) return r;
  DeviceGuard g(ctx->device);
  const int N = model->nx * model->ny;
  if ((r = ensure_site_scratch(ctx, N))) return r;
  if (!ctx->red && cudaMalloc(&ctx->red, reduce_scratch_doubles(0) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KPM_ENOMEM, "cudaMalloc failed");
  }
  cudaStream_t s = (cudaStream_t)stream;
  KPM_CU(launch_fields(*model, phi, params, mu, fields, ctx->wsite, s));
  if (w_out) KPM_CU(launch_sum(ctx->wsite, N, w_out, ctx->red, s));
  return KPM_OK;
}

int kpm_bounds(kpm_ctx* ctx, const kpm_model* model, const double* fields, double margin, double* ab,
               void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if ((r = check_dev(ctx, fields, "fields")) || (r = check_dev(ctx, ab, "ab"))) return r;
  if (!(margin >= 0.0)) return fail(ctx, KPM_EINVAL, "margin must be >= 0");
  DeviceGuard g(ctx->device);
  if (!ctx->red && cudaMalloc(&ctx->red, reduce_scratch_doubles(0) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KPM_ENOMEM, "cudaMalloc failed");
  }
  KPM_CU(launch_gershgorin(*model, fields, margin, ab, ctx->red, (cudaStream_t)stream));
  return KPM_OK;
}

int kpm_observables(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const double* fields,
                    const double* ab, double* obs, double* omega, void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if ((r = check_dev(ctx, fields, "fields")) || (r = check_dev(ctx, ab, "ab")) || (r = check_dev(ctx, obs, "obs")))
    return r;
  if (omega && (r = check_dev(ctx, omega, "omega"))) return r;
  DeviceGuard g(ctx->device);
  PassPlan pp;
  if ((r = plan_pass(ctx, model, opts, &pp))) return r;
  if ((r = ensure_pass_scratch(ctx, model, opts, pp))) return r;
  if (opts->flags & KPM_FLAG_PH_HALF) {
    if ((r = check_ph_sector(ctx, model, fields, ab, (cudaStream_t)stream))) return r;
  }
  void* tail = nullptr;
  ctx->tail_valid = false;
  if ((opts->flags & KPM_FLAG_KEEP_TAIL) && opts->M >= 2) {
    if (opts->precision == KPM_DF64 || opts->probe_p || (opts->flags & KPM_FLAG_PH_HALF))
      return fail(ctx, KPM_EINVAL, "KPM_FLAG_KEEP_TAIL: FP32 or FP64 unit-vector passes only");
    const int N = model->nx * model->ny;
    const size_t vec = (size_t)pp.cheb.D * pp.cheb.ldv * pp.elem;
    const int64_t nslab = (pp.c1 - pp.c0 + pp.width - 1) / pp.width;
    if ((r = ensure(ctx, &ctx->tail, &ctx->tail_bytes, 2 * (size_t)nslab * vec))) return r;
    if ((r = ensure(ctx, &ctx->tail_in, &ctx->tail_in_bytes, (26 * (size_t)N + 2) * sizeof(double)))) return r;
    cudaStream_t s = (cudaStream_t)stream;
    KPM_CU(cudaMemcpyAsync(ctx->tail_in, fields, 26 * (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    KPM_CU(cudaMemcpyAsync(ctx->tail_in + 26 * (size_t)N, ab, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    tail = ctx->tail;
  }
  r = enqueue_pass(ctx, model, opts, pp, fields, ab, obs, omega, (cudaStream_t)stream, false, nullptr, nullptr,
                   nullptr, nullptr, tail);
  if (r == KPM_OK && tail) {
    ctx->tail_valid = true;
    ctx->tail_model = *model;
    ctx->tail_opts = *opts;
    ctx->tail_width = pp.width;
    ctx->tail_c0 = pp.c0;
    ctx->tail_c1 = pp.c1;
  }
  return r;
}

int check_rmft_opts(kpm_ctx* ctx, const kpm_rmft_opts* ro) {
  if (!ro) return fail(ctx, KPM_EINVAL, "rmft opts is null");
  if (!(ro->alpha > 0.0 && ro->alpha <= 1.0 && ro->alpha_n > 0.0 && ro->alpha_n <= 1.0))
    return fail(ctx, KPM_EINVAL, "mixing must lie in (0, 1]");
  if (ro->anderson < 0 || ro->anderson > 16) return fail(ctx, KPM_EINVAL, "anderson must lie in 0..16");
  if (ro->sync_every < 0) return fail(ctx, KPM_EINVAL, "sync_every must be >= 0");
  return KPM_OK;
}

int rmft_prepare(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const double* phi,
                 const double* params, const double* mu_eff, double* fields, double* ab, double* mu_out,
                 void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if (!opts) return fail(ctx, KPM_EINVAL, "opts is null");
  if ((r = check_dev(ctx, phi, "phi")) || (r = check_dev(ctx, params, "params")) ||
      (r = check_dev(ctx, mu_eff, "mu_eff")) || (r = check_dev(ctx, fields, "fields")) ||
      (r = check_dev(ctx, ab, "ab")) || (r = check_dev(ctx, mu_out, "mu_out")))
    return r;
  if (!(opts->margin >= 0.0)) return fail(ctx, KPM_EINVAL, "margin must be >= 0");
  DeviceGuard g(ctx->device);
  const int N = model->nx * model->ny;
  if ((r = ensure_misc(ctx))) return r;
  if (!ctx->red && cudaMalloc(&ctx->red, reduce_scratch_doubles(0) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KPM_ENOMEM, "cudaMalloc failed");
  }
  cudaStream_t s = (cudaStream_t)stream;
  KPM_CU(launch_fields(*model, phi, params, 0.0, fields, nullptr, s));
  KPM_CU(launch_shift_eps(N, fields, mu_eff, ctx->misc + 6, mu_out, ctx->red, s));
  KPM_CU(launch_gershgorin(*model, fields, opts->margin, ab, ctx->red, s, (opts->flags & KPM_FLAG_PH_HALF) ? 1 : 0));
  return KPM_OK;
}

int rmft_update(kpm_ctx* ctx, const kpm_model* model, const kpm_rmft_opts* ropts, double* params, double* obs,
                double* mu_eff, double* stats_out, void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model)) || (r = check_rmft_opts(ctx, ropts))) return r;
  if (ropts->anderson != 0) return fail(ctx, KPM_EINVAL, "rmft_update mixes linearly (anderson must be 0)");
  if ((r = check_dev(ctx, params, "params")) || (r = check_dev(ctx, obs, "obs")) ||
      (r = check_dev(ctx, mu_eff, "mu_eff")) || (r = check_dev(ctx, stats_out, "stats_out")))
    return r;
  DeviceGuard g(ctx->device);
  if (!ctx->red && cudaMalloc(&ctx->red, reduce_scratch_doubles(0) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KPM_ENOMEM, "cudaMalloc failed");
  }
  KPM_CU(launch_update(model->nx * model->ny, params, obs, mu_eff, *ropts, stats_out, ctx->red, (cudaStream_t)stream));
  return KPM_OK;
}

int rmft_iterate(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const kpm_rmft_opts* ropts,
                 const double* phi, double* params, double* mu_eff, int n_iter, kpm_rmft_stats* stats,
                 void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if (!ropts || !phi || !params || !mu_eff) return fail(ctx, KPM_EINVAL, "null argument");
  if (n_iter < 0) return fail(ctx, KPM_EINVAL, "n_iter must be >= 0");
  if ((r = check_rmft_opts(ctx, ropts))) return r;
  DeviceGuard g(ctx->device);
  const int N = model->nx * model->ny;
  cudaStream_t s = (cudaStream_t)stream;
  PassPlan pp;
  if ((r = plan_pass(ctx, model, opts, &pp))) return r;
  if (pp.ranged) return fail(ctx, KPM_EINVAL, "rmft_iterate needs the whole lattice (site range 0, 0)");
  if ((r = ensure_site_scratch(ctx, N))) return r;
  if ((r = ensure_pass_scratch(ctx, model, opts, pp))) return r;
  if ((r = ensure_misc(ctx))) return r;
  AndersonState an;
  if (ropts->anderson > 0) {
    const size_t need = anderson_doubles(N, ropts->anderson) * sizeof(double);
    if (ctx->and_bytes < need) drop_graph(ctx);
    if ((r = ensure(ctx, &ctx->and_buf, &ctx->and_bytes, need))) return r;
    an = anderson_state(N, ropts->anderson, ctx->and_buf);
  }

  // host or device buffers: stage host ones through the context
  const bool params_dev = is_device_ptr(params);
  const bool phi_dev = is_device_ptr(phi);
  const bool mu_dev = is_device_ptr(mu_eff);
  double* dpar = params_dev ? params : ctx->dparams;
  const double* dphi = phi_dev ? phi : ctx->dphi;
  double* dmu = mu_dev ? mu_eff : ctx->misc + 7;
  if (!params_dev) KPM_CU(cudaMemcpyAsync(dpar, params, 26 * (size_t)N * sizeof(double), cudaMemcpyHostToDevice, s));
  if (!phi_dev) KPM_CU(cudaMemcpyAsync((void*)dphi, phi, 4 * (size_t)N * sizeof(double), cudaMemcpyHostToDevice, s));
  if (!mu_dev) KPM_CU(cudaMemcpyAsync(dmu, mu_eff, sizeof(double), cudaMemcpyHostToDevice, s));
  if (opts->flags & KPM_FLAG_PH_HALF) {
    // the half pass keeps the sector exactly (spin-down observables are copies)
    KPM_CU(launch_fields(*model, dphi, dpar, 0.0, ctx->fields, nullptr, s));
    if ((r = check_ph_sector(ctx, model, ctx->fields, nullptr, s))) return r;
  }

  kpm_ctx::Key key;
  memset(&key, 0, sizeof(key));
  key.m = *model;
  key.o = *opts;
  key.r = *ropts;
  key.phi = dphi;
  key.params = dpar;
  key.mu_eff = dmu;
  if (!ctx->key_valid || !same_key(key, ctx->key)) {
    drop_graph(ctx);
    // capture one iteration on the context's stream
    cudaStream_t c = ctx->cap;
    KPM_CU(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal));
    double* ab = ctx->misc;
    int rr = KPM_OK;
    cudaError_t e = launch_fields(*model, dphi, dpar, 0.0, ctx->fields, nullptr, c);
    if (e == cudaSuccess) e = launch_shift_eps(N, ctx->fields, dmu, ctx->misc + 6, ctx->misc + 2, ctx->red, c);
    if (e == cudaSuccess)
      e = launch_gershgorin(*model, ctx->fields, opts->margin, ab, ctx->red, c, (opts->flags & KPM_FLAG_PH_HALF) ? 1 : 0);
    int npass = 0, nrec = 0;
    double nbytes = 0.0;
    if (e == cudaSuccess)
      rr = enqueue_pass(ctx, model, opts, pp, ctx->fields, ab, ctx->obs, ctx->misc + 3, c, true, &npass, &nrec,
                        &nbytes);
    // fields 1, mean-shift 3, bounds 2, pass, update 4 (Anderson: 7)
    ctx->launches = 1 + 3 + 2 + npass + (ropts->anderson > 0 ? 7 : 4);
    ctx->rec_launches = nrec;
    ctx->rec_bytes = nbytes;
    if (e == cudaSuccess && rr == KPM_OK)
      e = launch_update(N, dpar, ctx->obs, dmu, *ropts, ctx->misc + 4, ctx->red, c, ctx->misc + kRec, ctx->misc,
                        ropts->anderson > 0 ? &an : nullptr);
    if (e == cudaSuccess && rr == KPM_OK)
      e = cudaMemcpyAsync(ctx->host_misc + kRec, ctx->misc + kRec, 16 * sizeof(double), cudaMemcpyDeviceToHost, c);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c, &graph);
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(ctx, e, "capture of the RMFT iteration");
    }
    if (rr != KPM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rr;
    }
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->graph = nullptr;
      return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    ctx->key = key;
    ctx->key_valid = true;
  }

  kpm_rmft_stats st;
  memset(&st, 0, sizeof(st));
  int status = KPM_OK;
  st.kernel_launches = ctx->launches;
  st.recursion_launches = ctx->rec_launches;
  // a fresh record (iteration count, frozen flag, Anderson history length)
  // and, for Anderson mixing, an empty history
  KPM_CU(cudaMemsetAsync(ctx->misc + kRec, 0, 16 * sizeof(double), s));
  if (ropts->anderson > 0)
    KPM_CU(cudaMemsetAsync(an.dX, 0, 2 * (size_t)ropts->anderson * (26 * (size_t)N + 1) * sizeof(double), s));
  const int group = std::max(1, ropts->sync_every);
  for (int done = 0; done < n_iter;) {
    const int k = std::min(group, n_iter - done);
    for (int j = 0; j < k; ++j) KPM_CU(cudaGraphLaunch(ctx->graph, s));
    KPM_CU(cudaStreamSynchronize(s));
    done += k;
    if (ctx->rec_launches > 0) {
      float ms = 0.f;
      KPM_CU(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
      st.recursion_ms += (double)ms * k;
      st.recursion_bytes += ctx->rec_bytes * k;
    }
    const double* h = ctx->host_misc + kRec;
    st.a = h[0];
    st.b = h[1];
    st.mu = h[2];
    st.omega = h[3];
    st.residual = h[4];
    st.density_error = h[5];
    st.iterations = (int)h[6];
    if (!(st.residual == st.residual) || !(st.omega == st.omega) || st.residual > 1e300) {
      status = device_fault_status(ctx);
      if (status == KPM_OK) status = fail(ctx, KPM_ENONFINITE, "non-finite order parameters in the RMFT iteration");
      break;
    }
    st.converged = st.residual < ropts->tol && fabs(st.density_error) < ropts->tol;
    if (st.converged) break;
  }
  if (status == KPM_OK && ropts->strict && !st.converged && n_iter > 0)
    status = fail(ctx, KPM_ENOTCONV, "rmft_iterate: tol not met within n_iter iterations");
  if (!params_dev) KPM_CU(cudaMemcpyAsync(params, dpar, 26 * (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!mu_dev) KPM_CU(cudaMemcpyAsync(mu_eff, dmu, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!params_dev || !mu_dev) KPM_CU(cudaStreamSynchronize(s));
  if (stats) *stats = st;
  return status;
}

int kpm_backward(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const double* fields,
                 const double* ab, const double* grad_obs, double grad_omega, double* grad_fields,
                 const double* phi, const double* params, double* grad_phi, int ckpt_every, void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if ((r = check_dev(ctx, fields, "fields")) || (r = check_dev(ctx, ab, "ab")) ||
      (r = check_dev(ctx, grad_obs, "grad_obs")) || (r = check_dev(ctx, grad_fields, "grad_fields")))
    return r;
  if (grad_phi && ((r = check_dev(ctx, grad_phi, "grad_phi")) || (r = check_dev(ctx, phi, "phi")) ||
                   (r = check_dev(ctx, params, "params"))))
    return r;
  if (!opts) return fail(ctx, KPM_EINVAL, "opts is null");
  if (ckpt_every < KPM_REGENERATE) return fail(ctx, KPM_EINVAL, "ckpt_every must be >= 0 or KPM_REGENERATE");
  DeviceGuard g(ctx->device);
  const int N = model->nx * model->ny;
  const int64_t D = 2 * (int64_t)N;
  const int M = opts->M;
  const bool regen = ckpt_every == KPM_REGENERATE;
  int seg = ckpt_every > 0 ? ckpt_every : (int)lround(sqrt((double)M));
  if (seg < 2) seg = 2;
  // checkpoints: segments serving m in [k seg + 1, (k+1) seg], each with two
  // checkpoints; regenerating: no checkpoints, only the lambda pair here (the
  // alpha pair lives in the recursion slabs)
  const int K = regen ? 0 : (M >= 2 ? (M - 1 + seg - 1) / seg : 0);
  const int nvec = regen ? 2 : 2 * K + seg + 2;

  if (opts->precision == KPM_DF64) return fail(ctx, KPM_EINVAL, "KPM_DF64: not supported by kpm_backward");
  if (opts && (opts->flags & KPM_FLAG_PH_HALF)) return fail(ctx, KPM_EINVAL, "KPM_FLAG_PH_HALF: not supported by kpm_backward");
  if (opts && opts->probe_p) return fail(ctx, KPM_EINVAL, "probing: not supported by kpm_backward");
  // slab width from the budget over all adjoint slab vectors (plus the forward pair);
  // the adjoint steps one moment per launch (its recomputed segments are stored)
  kpm_opts o = *opts;
  o.flags &= ~(KPM_FLAG_DOUBLE_STEP | KPM_FLAG_KEEP_TAIL);
  const size_t elem = o.precision == KPM_FP32 ? 8 : 16;
  // regenerating from the tail of the last kpm_observables: same model, same
  // pass options and the same fields and ab (compared on the device below)
  bool use_tail = false;
  if (regen && ctx->tail_valid && M >= 2) {
    kpm_opts t = ctx->tail_opts;
    t.flags &= ~(KPM_FLAG_DOUBLE_STEP | KPM_FLAG_KEEP_TAIL);
    kpm_opts q = o;
    if (q.block_width == 0) q.block_width = t.block_width;
    use_tail = memcmp(&ctx->tail_model, model, sizeof(kpm_model)) == 0 && memcmp(&t, &q, sizeof(kpm_opts)) == 0;
    if (use_tail) {
      int same = 0;
      if ((r = ensure_misc(ctx))) return r;
      KPM_CU(launch_same_doubles(fields, ctx->tail_in, 26 * (int64_t)N, ab, ctx->tail_in + 26 * (size_t)N, 2,
                                 reinterpret_cast<int*>(ctx->misc + 14), reinterpret_cast<int*>(ctx->host_misc + 14),
                                 &same, (cudaStream_t)stream));
      use_tail = same != 0;
    }
    if (use_tail) o.block_width = (int)ctx->tail_width;  // the forward's slabs
  }
  // unit columns of the pass (all D, or those of the site range)
  const int64_t ncol = (o.site_begin != 0 || o.site_end != 0) ? 2 * ((int64_t)o.site_end - o.site_begin) : D;
  if (o.block_width == 0 && ncol > 0) {
    const int64_t fit = (int64_t)(ctx->budget / ((uint64_t)(nvec + 2) * D * elem));
    o.block_width = (int)balanced_width(ncol, std::max<int64_t>(1, std::min<int64_t>(ncol, fit)));
  }
  PassPlan pp;
  if ((r = plan_pass(ctx, model, &o, &pp))) return r;
  if ((r = ensure_pass_scratch(ctx, model, &o, pp))) return r;
  const ChebPlan& p = pp.cheb;
  const size_t vbytes = (size_t)D * p.ldv * elem;
  if (use_tail) {
    // the tail is read slab by slab: only with the forward pass's exact slabs
    const int64_t nslab = (pp.c1 - pp.c0 + pp.width - 1) / pp.width;
    use_tail = pp.width == ctx->tail_width && pp.c0 == ctx->tail_c0 && pp.c1 == ctx->tail_c1 &&
               (size_t)(2 * nslab) * vbytes <= ctx->tail_bytes;
  }
  if ((r = ensure(ctx, &ctx->bwd, &ctx->bwd_bytes, vbytes * (size_t)nvec))) return r;
  const int groups = grad_groups(p, o.precision);
  const size_t gbytes = (size_t)D * 13 * sizeof(double2);  // G, then the column sets' partial sums
  if ((r = ensure(ctx, &ctx->Gacc, &ctx->Gacc_bytes, gbytes * (size_t)(groups + 1)))) return r;
  double2* Gpart = ctx->Gacc + (size_t)D * 13;
  if ((r = ensure(ctx, &ctx->wseed, &ctx->wseed_bytes, (size_t)D * kSlots * sizeof(double2)))) return r;
  char* base = static_cast<char*>(ctx->bwd);
  auto ckpt = [&](int k) { return (void*)(base + vbytes * (size_t)k); };
  auto segv = [&](int j) { return (void*)(base + vbytes * (size_t)(2 * K + j)); };
  // the lambda pair: the last two of the nvec vectors (checkpoints and the
  // segment first when checkpointing; alone when regenerating)
  void* lamA = base + vbytes * (size_t)(nvec - 2);
  void* lamB = base + vbytes * (size_t)(nvec - 1);

  cudaStream_t s = (cudaStream_t)stream;
  const int prec = o.precision;
  void* A = ctx->slab[0];
  void* B = ctx->slab[1];
  KPM_CU(launch_coefficients(M, ab, ctx->am, ctx->ao, s, 0, o.temperature));
  if (prec == KPM_FP32)
    KPM_CU(launch_scale_table_f32(*model, fields, ab, (float2*)ctx->table, s));
  else
    KPM_CU(launch_scale_table_f64(*model, fields, ab, (double2*)ctx->table, s));
  // seeds of the columns outside the site range are zero: their backward
  // vectors stay zero, so they add nothing where a slab runs past the range
  KPM_CU(launch_seed_weights(model->nx, model->ny, grad_obs, ab, grad_omega, ctx->wseed, s, pp.sb, pp.se));
  KPM_CU(cudaMemsetAsync(Gpart, 0, gbytes * (size_t)groups, s));
  const double* am = ctx->am;
  const double* ao = ctx->ao;

  // Reversible recursion: alpha_{m-1} = 2 h~ alpha_m - alpha_{m+1} (Eq. alpha
  // run backwards), so from the last two vectors every earlier one is
  // regenerated by one more step, in the order the backward sweep needs them.
  for (int64_t s0 = pp.c0; regen && s0 < pp.c1 && M >= 2; s0 += pp.width) {
    void* hi = A;  // alpha_{M-1}
    void* lo = B;  // alpha_{M-2}
    if (use_tail) {
      const char* t = static_cast<const char*>(ctx->tail) + (size_t)(2 * ((s0 - pp.c0) / pp.width)) * vbytes;
      KPM_CU(cudaMemcpyAsync(lo, t, vbytes, cudaMemcpyDeviceToDevice, s));
      KPM_CU(cudaMemcpyAsync(hi, t + vbytes, vbytes, cudaMemcpyDeviceToDevice, s));
    } else {
      // forward sweep keeping only the last pair: X0 = alpha_{mm-1}, X1 = alpha_mm
      void* X0 = A;
      void* X1 = B;
      KPM_CU(launch_cheb_init(p, prec, X0, s0, ctx->acc, am, ao, s));
      KPM_CU(launch_cheb_step(p, prec, ctx->table, X0, X1, s0, nullptr, am, ao, 0, 0, s));
      for (int mm = 1; mm + 1 <= M - 1; ++mm) {
        KPM_CU(launch_cheb_step(p, prec, ctx->table, X1, X0, s0, nullptr, am, ao, mm, 1, s));
        std::swap(X0, X1);
      }
      hi = X1;
      lo = X0;
    }
    void* lcur = lamA;
    void* lnxt = lamB;
    KPM_CU(cudaMemsetAsync(lcur, 0, vbytes, s));
    KPM_CU(cudaMemsetAsync(lnxt, 0, vbytes, s));
    for (int m = M - 1; m >= 1; --m) {
      if (m < M - 1) {
        // alpha_{m-1} = 2 h~ alpha_m - alpha_{m+1}, in place over alpha_{m+1}
        KPM_CU(launch_cheb_step(p, prec, ctx->table, lo, hi, s0, nullptr, am, ao, 0, 1, s));
        std::swap(hi, lo);
      }
      // lnxt <- 2 h~ lambda_{m+1} - lambda_{m+2} + c_m = lambda_m
      KPM_CU(launch_cheb_step(p, prec, ctx->table, lcur, lnxt, s0, nullptr, am, ao, 0, 1, s));
      KPM_CU(launch_seed_scatter(p, prec, lnxt, s0, ctx->wseed, am, ao, m, s));
      KPM_CU(launch_grad_accum(p, prec, lnxt, lo, m == 1 ? 1.0 : 2.0, Gpart, s));
      std::swap(lcur, lnxt);
    }
  }

  for (int64_t s0 = pp.c0; !regen && s0 < pp.c1 && M >= 2; s0 += pp.width) {
    // forward, writing the checkpointed vectors (alpha_{k seg}, alpha_{k seg + 1})
    // in place and stepping through the two temporaries otherwise
    auto ckpt_slot = [&](int idx) -> void* {
      if (idx % seg == 0 && idx / seg < K) return ckpt(2 * (idx / seg));
      if (idx % seg == 1 && idx / seg < K) return ckpt(2 * (idx / seg) + 1);
      return nullptr;
    };
    KPM_CU(launch_cheb_init(p, prec, ckpt(0), s0, ctx->acc, am, ao, s));
    KPM_CU(launch_cheb_step(p, prec, ctx->table, ckpt(0), ckpt(1), s0, nullptr, am, ao, 0, 0, s));
    const void* a_prev = ckpt(0);
    const void* a_cur = ckpt(1);
    const int last_needed = (K - 1) * seg + 1;  // highest checkpointed index
    for (int mm = 1; mm + 1 <= last_needed; ++mm) {
      void* dest = ckpt_slot(mm + 1);
      if (!dest) {
        if (a_prev == A || a_prev == B) dest = const_cast<void*>(a_prev);  // in place over alpha_{mm-1}
        else dest = (a_cur == A) ? B : A;
      }
      KPM_CU(launch_cheb_step(p, prec, ctx->table, a_cur, dest, s0, nullptr, am, ao, mm, 1, s, a_prev));
      a_prev = a_cur;
      a_cur = dest;
    }
    // backward: lambda_{m+1} in `lcur`, lambda_{m+2} in `lnxt`, both zero above M-1
    void* lcur = lamA;
    void* lnxt = lamB;
    KPM_CU(cudaMemsetAsync(lcur, 0, vbytes, s));
    KPM_CU(cudaMemsetAsync(lnxt, 0, vbytes, s));
    std::vector<const void*> segp(seg);
    for (int k = K - 1; k >= 0; --k) {
      const int m_hi = std::min((k + 1) * seg, M - 1);
      const int m_lo = k * seg + 1;
      // alpha_{k seg} .. alpha_{m_hi - 1}: two checkpoints, then out-of-place steps
      const int nseg = m_hi - k * seg;
      segp[0] = ckpt(2 * k);
      if (nseg > 1) segp[1] = ckpt(2 * k + 1);
      for (int j = 2; j < nseg; ++j) {
        KPM_CU(launch_cheb_step(p, prec, ctx->table, segp[j - 1], segv(j), s0, nullptr, am, ao, 0, 1, s, segp[j - 2]));
        segp[j] = segv(j);
      }
      for (int m = m_hi; m >= m_lo; --m) {
        // lnxt <- 2 h~ lambda_{m+1} - lambda_{m+2} + c_m = lambda_m
        KPM_CU(launch_cheb_step(p, prec, ctx->table, lcur, lnxt, s0, nullptr, am, ao, 0, 1, s));
        KPM_CU(launch_seed_scatter(p, prec, lnxt, s0, ctx->wseed, am, ao, m, s));
        KPM_CU(launch_grad_accum(p, prec, lnxt, segp[m - 1 - k * seg], m == 1 ? 1.0 : 2.0, Gpart, s));
        std::swap(lcur, lnxt);
      }
    }
  }
  KPM_CU(launch_grad_reduce(D, groups, Gpart, ctx->Gacc, s));
  KPM_CU(launch_grad_fields(model->nx, model->ny, ctx->Gacc, ab, grad_fields, s));
  if (grad_phi) KPM_CU(launch_phi_grad(*model, phi, params, grad_fields, grad_phi, s));
  return KPM_OK;
}

int kpm_order_parameters(kpm_ctx* ctx, const kpm_model* model, const double* phi, const double* params,
                         double* delta_out, double* mag_out, void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if ((r = check_dev(ctx, phi, "phi")) || (r = check_dev(ctx, params, "params")) ||
      (r = check_dev(ctx, delta_out, "delta_out")) || (r = check_dev(ctx, mag_out, "mag_out")))
    return r;
  DeviceGuard g(ctx->device);
  KPM_CU(launch_order_parameters(*model, phi, params, delta_out, mag_out, (cudaStream_t)stream));
  return KPM_OK;
}

int kpm_ldos(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const double* fields, const double* ab,
             const double* params, int n_omega, const double* omega, double gamma_alpha, double gamma0, double* ldos,
             void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if ((r = check_dev(ctx, fields, "fields")) || (r = check_dev(ctx, ab, "ab")) || (r = check_dev(ctx, ldos, "ldos")))
    return r;
  if (params && (r = check_dev(ctx, params, "params"))) return r;
  if (!opts || !omega || n_omega < 1) return fail(ctx, KPM_EINVAL, "bad LDOS arguments");
  if (!(gamma0 > 0.0) || !(gamma_alpha >= 0.0)) return fail(ctx, KPM_EINVAL, "need gamma0 > 0 and gamma_alpha >= 0");
  if (opts->flags & KPM_FLAG_PH_HALF) return fail(ctx, KPM_EINVAL, "KPM_FLAG_PH_HALF: the LDOS needs both Nambu rows");
  if (opts->precision == KPM_DF64) return fail(ctx, KPM_EINVAL, "KPM_DF64: not supported by kpm_ldos");
  if (opts->site_begin || opts->site_end) return fail(ctx, KPM_EINVAL, "site range: not supported by kpm_ldos");
  DeviceGuard g(ctx->device);
  const int N = model->nx * model->ny;
  const int64_t D = 2 * (int64_t)N;
  const int M = opts->M;
  kpm_opts o = *opts;
  o.flags &= ~KPM_FLAG_DOUBLE_STEP;  // one step per launch
  if ((r = ensure_site_scratch(ctx, N))) return r;
  PassPlan pp;
  if ((r = plan_pass(ctx, model, &o, &pp))) return r;
  if ((r = ensure_pass_scratch(ctx, model, &o, pp))) return r;
  // scratch: record M x D, coefficients 2 x n_omega x M, weights 2N, frequencies n_omega
  const size_t rec_n = (size_t)M * D, c_n = 2 * (size_t)n_omega * M;
  const size_t need = (rec_n + c_n + 2 * (size_t)N + (size_t)n_omega) * sizeof(double);
  if ((r = ensure(ctx, &ctx->ldos_buf, &ctx->ldos_buf_bytes, need))) return r;
  double* rec = ctx->ldos_buf;
  double* C = rec + rec_n;
  double* wgt = C + c_n;
  double* om = wgt + 2 * (size_t)N;
  if (!ctx->cublas && !(ctx->cublas = cublas_create())) return fail(ctx, KPM_ECUDA, "cublasCreate failed");
  cudaStream_t s = (cudaStream_t)stream;
  KPM_CU(cudaMemcpyAsync(om, omega, n_omega * sizeof(double),
                         is_device_ptr(omega) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if ((r = enqueue_pass(ctx, model, &o, pp, fields, ab, ctx->obs, nullptr, s, false, nullptr, nullptr, nullptr, rec)))
    return r;
  if (params) KPM_CU(launch_gt_weights(*model, params, wgt, s));
  KPM_CU(launch_ldos_coefficients(M, n_omega, om, gamma_alpha, gamma0, ab, C, s));
  const char* err = ldos_contract(ctx->cublas, M, n_omega, N, C, rec, ldos, params ? wgt : nullptr, s);
  if (err) return fail(ctx, KPM_ECUDA, err);
  return KPM_OK;
}

int rmft_iterate_batched(kpm_ctx* ctx, int ncell, const kpm_model* models, const kpm_opts* opts,
                         const kpm_rmft_opts* ropts, const double* const* phis, double* const* params,
                         double* mu_eff, int n_iter, kpm_rmft_stats* stats, void* stream) {
  if (!ctx) return KPM_EINVAL;
  if (ncell < 1 || ncell > 4096 || !models || !opts || !ropts || !phis || !params || !mu_eff || n_iter < 0)
    return fail(ctx, KPM_EINVAL, "bad batch arguments");
  int r;
  for (int c = 0; c < ncell; ++c) {
    if ((r = check_model(ctx, &models[c]))) return r;
    if ((r = check_dev(ctx, phis[c], "phis[c]")) || (r = check_dev(ctx, params[c], "params[c]"))) return r;
    if (!(ropts[c].alpha > 0.0 && ropts[c].alpha <= 1.0 && ropts[c].alpha_n > 0.0 && ropts[c].alpha_n <= 1.0))
      return fail(ctx, KPM_EINVAL, "mixing must lie in (0, 1]");
  }
  if ((r = check_dev(ctx, mu_eff, "mu_eff"))) return r;
  if (opts->flags & KPM_FLAG_PH_HALF) return fail(ctx, KPM_EINVAL, "KPM_FLAG_PH_HALF: not supported by the batched call");
  if (opts->probe_p) return fail(ctx, KPM_EINVAL, "probing: not supported by the batched call");
  if (opts->site_begin || opts->site_end) return fail(ctx, KPM_EINVAL, "site range: not supported by the batched call");
  for (int c = 0; c < ncell; ++c)
    if ((r = check_rmft_opts(ctx, &ropts[c]))) return r;
    else if (ropts[c].anderson || ropts[c].sync_every > 1)
      return fail(ctx, KPM_EINVAL, "the batched call mixes linearly and reads every iteration");
  if (opts->M < 1 || (opts->precision != KPM_FP32 && opts->precision != KPM_FP64))
    return fail(ctx, KPM_EINVAL, "bad opts");
  DeviceGuard g(ctx->device);
  const int M = opts->M, prec = opts->precision;
  const size_t elem = prec == KPM_FP32 ? 8 : 16;

  // shape classes (cells of equal nx, ny share one batched launch per step)
  std::map<std::pair<int, int>, int> cls_of;
  std::vector<std::vector<int>> members;
  for (int c = 0; c < ncell; ++c) {
    auto key = std::make_pair(models[c].nx, models[c].ny);
    auto it = cls_of.find(key);
    if (it == cls_of.end()) {
      it = cls_of.emplace(key, (int)members.size()).first;
      members.emplace_back();
    }
    members[it->second].push_back(c);
  }
  for (auto& v : members)
    if ((int)v.size() > kMaxBatch && prec == KPM_FP32) return fail(ctx, KPM_EINVAL, "more than 64 cells of one shape");
  std::vector<ChebPlan> plans(members.size());
  for (size_t k = 0; k < members.size(); ++k) {
    const kpm_model& m0 = models[members[k][0]];
    const int64_t D = 2 * (int64_t)m0.nx * m0.ny;
    plans[k] = plan_cheb(m0.nx, m0.ny, D, prec, opts->cols_per_block, opts->band_rows);
    if (plans[k].cb == 0) return fail(ctx, KPM_EINVAL, "lattice row too wide for the shared-memory window");
    // spread one step over the whole batch: y bands so that every cell fills its share
    const int64_t chunks = plans[k].ldv / plans[k].cb;
    const int64_t want = std::max<int64_t>(1, 4 * 152 / (int64_t)std::max<size_t>(1, members[k].size()));
    const int yb = (int)std::min<int64_t>(m0.ny, std::max<int64_t>(1, (want + chunks - 1) / chunks));
    plans[k].ylen = std::max(1, (m0.ny + yb - 1) / yb);
    cudaError_t e = prec == KPM_FP32 ? cheb_prepare_batched(plans[k]) : cheb_prepare(plans[k], prec);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "prepare");
  }

  // FP32 shape classes whose band of a cell fits shared memory run the
  // persistent recursion (one launch for all of them, all M moments on chip);
  // the others keep one batched step launch per moment
  std::vector<char> persist(members.size(), 0);
  size_t psmem = 0;
  int pclusters = 0;
  if (prec == KPM_FP32 && M >= 1) {
    for (size_t k = 0; k < members.size(); ++k) {
      const kpm_model& m0 = models[members[k][0]];
      const size_t sm = persist_smem_bytes(m0.nx, m0.ny);
      if (sm <= 227 * 1024) {
        persist[k] = 1;
        psmem = std::max(psmem, sm);
      }
    }
    if (psmem > 0) {
      cudaError_t e = persist_prepare(psmem, &pclusters);
      if (e != cudaSuccess) {
        cudaGetLastError();
        std::fill(persist.begin(), persist.end(), 0);
        psmem = 0;
      }
    }
  }

  // per-cell scratch, one allocation per cell
  auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
  bool realloc = (int)ctx->cells.size() != ncell;
  std::vector<size_t> need(ncell);
  for (int c = 0; c < ncell; ++c) {
    const int N = models[c].nx * models[c].ny;
    const int64_t D = 2 * (int64_t)N;
    const int k = cls_of[std::make_pair(models[c].nx, models[c].ny)];
    // (cells of the persistent recursion keep their vectors in shared memory: no slabs)
    need[c] = al(26 * (size_t)N * 8) * 2 + al((size_t)M * 8) * 2 + al(16 * 8) + al((size_t)D * kSlots * 16) +
              al((size_t)N * table_bytes_per_site(prec)) + (persist[k] ? 0 : 2 * al((size_t)D * plans[k].ldv * elem));
    if (!realloc && ctx->cells[c].bytes < need[c]) realloc = true;
  }
  if (realloc) {
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    ctx->bgraph = nullptr;
    ctx->bkey.clear();
    for (auto& c : ctx->cells)
      if (c.mem) cudaFree(c.mem);
    ctx->cells.assign(ncell, kpm_ctx::Cell());
    for (int c = 0; c < ncell; ++c) {
      if (cudaMalloc(&ctx->cells[c].mem, need[c]) != cudaSuccess) {
        cudaGetLastError();
        ctx->cells[c].mem = nullptr;
        return fail(ctx, KPM_ENOMEM, "cudaMalloc of batch scratch failed");
      }
      ctx->cells[c].bytes = need[c];
    }
  }
  for (int c = 0; c < ncell; ++c) {
    const int N = models[c].nx * models[c].ny;
    const int64_t D = 2 * (int64_t)N;
    const int k = cls_of[std::make_pair(models[c].nx, models[c].ny)];
    char* b = static_cast<char*>(ctx->cells[c].mem);
    kpm_ctx::Cell& C = ctx->cells[c];
    C.fields = (double*)b; b += al(26 * (size_t)N * 8);
    C.obs = (double*)b; b += al(26 * (size_t)N * 8);
    C.am = (double*)b; b += al((size_t)M * 8);
    C.ao = (double*)b; b += al((size_t)M * 8);
    C.misc = (double*)b; b += al(16 * 8);
    C.acc = (double2*)b; b += al((size_t)D * kSlots * 16);
    C.table = b; b += al((size_t)N * table_bytes_per_site(prec));
    if (persist[k]) {
      C.A = C.B = nullptr;
    } else {
      C.A = b; b += al((size_t)D * plans[k].ldv * elem);
      C.B = b;
    }
    C.cls = k;
  }
  if (!ctx->bred && cudaMalloc(&ctx->bred, reduce_scratch_doubles(0) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KPM_ENOMEM, "cudaMalloc failed");
  }
  if (ctx->bhost_n < (size_t)ncell * 16) {
    if (ctx->bhost) cudaFreeHost(ctx->bhost);
    ctx->bhost = nullptr;
    if (cudaMallocHost(&ctx->bhost, (size_t)ncell * 16 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, KPM_ENOMEM, "cudaMallocHost failed");
    }
    ctx->bhost_n = (size_t)ncell * 16;
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    ctx->bgraph = nullptr;
    ctx->bkey.clear();
  }
  while (ctx->fork.size() < members.size()) {
    cudaStream_t st;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, KPM_ECUDA, "stream creation failed");
    }
    ctx->fork.push_back(st);
    ctx->fork_ev.push_back(ev);
  }
  if (!ctx->join_ev && cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, KPM_ECUDA, "event creation failed");
  }

  // graph key: everything the captured work depends on
  std::vector<char> key;
  auto put = [&](const void* p, size_t n) { key.insert(key.end(), (const char*)p, (const char*)p + n); };
  put(&ncell, sizeof(ncell));
  put(models, sizeof(kpm_model) * ncell);
  put(opts, sizeof(kpm_opts));
  put(ropts, sizeof(kpm_rmft_opts) * ncell);
  put(phis, sizeof(double*) * ncell);
  put(params, sizeof(double*) * ncell);
  put(&mu_eff, sizeof(mu_eff));
  if (!ctx->bgraph || key != ctx->bkey) {
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    ctx->bgraph = nullptr;
    cudaStream_t c0 = ctx->cap;
    // per shape class: the cells' pointers and, for the TMA-staged step, the
    // tensor maps of their slabs, uploaded before the capture (the graph
    // reads them from device memory on every replay)
    std::vector<BatchPtrs> bps(members.size());
    std::vector<const void*> maps_of(members.size(), nullptr);
    for (size_t k = 0; k < members.size(); ++k) {
      BatchPtrs& bp = bps[k];
      memset(&bp, 0, sizeof(bp));
      for (size_t z = 0; z < members[k].size(); ++z) {
        kpm_ctx::Cell& C = ctx->cells[members[k][z]];
        bp.A[z] = C.A;
        bp.B[z] = C.B;
        bp.table[z] = C.table;
        bp.acc[z] = C.acc;
        bp.am[z] = C.am;
        bp.ao[z] = C.ao;
      }
    }
    if (prec == KPM_FP32) {
      while (ctx->bmaps.size() < members.size()) {
        void* d = nullptr;
        if (cudaMalloc(&d, batch_maps_bytes(kMaxBatch)) != cudaSuccess) {
          cudaGetLastError();
          return fail(ctx, KPM_ENOMEM, "cudaMalloc of the batch tensor maps failed");
        }
        ctx->bmaps.push_back(d);
      }
      KPM_CU(cudaStreamSynchronize(c0));  // no replay of an older graph still reads the maps
      for (size_t k = 0; k < members.size(); ++k) {
        if (plans[k].tma_rows == 0 || persist[k]) continue;
        const int nz = (int)members[k].size();
        std::vector<CUtensorMap> host((size_t)2 * nz);
        KPM_CU(encode_batch_maps(plans[k], nz, bps[k], host.data()));
        KPM_CU(cudaMemcpy(ctx->bmaps[k], host.data(), batch_maps_bytes(nz), cudaMemcpyHostToDevice));
        maps_of[k] = ctx->bmaps[k];
      }
    }
    // persistent recursion: the cell table and the work items, longest first
    // (an item's time grows with its cell's band, nx ceil(ny / kPClu) sites),
    // uploaded before the capture like the tensor maps
    int nitems = 0, nx_max = 0, nclu = 0;
    PCell* d_cells = nullptr;
    PItem* d_items = nullptr;
    int* d_counter = nullptr;
    void* d_xbuf = nullptr;
    double pbytes = 0.0;
    if (psmem > 0) {
      std::vector<PCell> hc(ncell);
      std::vector<PItem> hi;
      const int q = persist_columns();
      for (int c = 0; c < ncell; ++c) {
        kpm_ctx::Cell& C = ctx->cells[c];
        hc[c] = PCell{models[c].nx, models[c].ny, (const float2*)C.table, C.acc, C.am, C.ao};
        if (!persist[C.cls]) continue;
        const int64_t D = 2 * (int64_t)models[c].nx * models[c].ny;
        nx_max = std::max(nx_max, models[c].nx);
        for (int64_t q0 = 0; q0 < D; q0 += q) hi.push_back(PItem{c, (int)q0});
        pbytes += 24.0 * (double)D * (double)D * (double)std::max(0, M - 1);
      }
      std::stable_sort(hi.begin(), hi.end(), [&](const PItem& a, const PItem& b) {
        auto cost = [&](const PItem& t) {
          const kpm_model& m = models[t.cell];
          return (int64_t)m.nx * ((m.ny + kPClu - 1) / kPClu);
        };
        return cost(a) > cost(b);
      });
      nitems = (int)hi.size();
      nclu = std::max(1, std::min(pclusters, nitems));
      const size_t xoff = al(sizeof(PCell) * ncell) + al(sizeof(PItem) * std::max(1, nitems)) + 256;
      const size_t need = xoff + persist_exchange_bytes(nclu, nx_max);
      KPM_CU(cudaStreamSynchronize(c0));  // no replay of an older graph still reads the tables
      if ((r = ensure(ctx, &ctx->pbuf, &ctx->pbuf_bytes, need))) return r;
      char* pb = static_cast<char*>(ctx->pbuf);
      d_cells = reinterpret_cast<PCell*>(pb);
      d_items = reinterpret_cast<PItem*>(pb + al(sizeof(PCell) * ncell));
      d_counter = reinterpret_cast<int*>(pb + al(sizeof(PCell) * ncell) + al(sizeof(PItem) * std::max(1, nitems)));
      d_xbuf = pb + xoff;
      KPM_CU(cudaMemcpy(d_cells, hc.data(), sizeof(PCell) * ncell, cudaMemcpyHostToDevice));
      if (nitems) KPM_CU(cudaMemcpy(d_items, hi.data(), sizeof(PItem) * nitems, cudaMemcpyHostToDevice));
      for (int k = 0; k < 2; ++k)
        if (!ctx->pev[k] && cudaEventCreate(&ctx->pev[k]) != cudaSuccess) {
          cudaGetLastError();
          return fail(ctx, KPM_ECUDA, "event creation failed");
        }
    }
    ctx->p_bytes = pbytes;
    ctx->p_launched = nitems > 0;

    KPM_CU(cudaStreamBeginCapture(c0, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const char* where = "";
#define KPM_TRY(expr)        \
  do {                       \
    if (e == cudaSuccess) {  \
      e = (expr);            \
      if (e != cudaSuccess) where = #expr; \
    }                        \
  } while (0)
    for (int c = 0; c < ncell; ++c) {
      kpm_ctx::Cell& C = ctx->cells[c];
      const kpm_model& m = models[c];
      const int N = m.nx * m.ny;
      const ChebPlan& p = plans[C.cls];
      KPM_TRY(launch_fields(m, phis[c], params[c], 0.0, C.fields, nullptr, c0));
      KPM_TRY(launch_shift_eps(N, C.fields, mu_eff + c, C.misc + 6, C.misc + 2, ctx->bred, c0));
      KPM_TRY(launch_gershgorin(m, C.fields, opts->margin, C.misc, ctx->bred, c0));
      KPM_TRY(launch_coefficients(M, C.misc, C.am, C.ao, c0, 0, opts->temperature));
      if (prec == KPM_FP32)
        KPM_TRY(launch_scale_table_f32(m, C.fields, C.misc, (float2*)C.table, c0));
      else
        KPM_TRY(launch_scale_table_f64(m, C.fields, C.misc, (double2*)C.table, c0));
      if (!persist[C.cls]) KPM_TRY(launch_cheb_init(p, prec, C.A, 0, C.acc, C.am, C.ao, c0));
    }
    // recursion: one chain per shape class on its own stream
    KPM_TRY(cudaEventRecord(ctx->join_ev, c0));
    for (size_t k = 0; k < members.size() && M >= 2; ++k) {
      if (persist[k]) continue;
      cudaStream_t sk = ctx->fork[k];
      KPM_TRY(cudaStreamWaitEvent(sk, ctx->join_ev, 0));
      const ChebPlan& p = plans[k];
      if (prec == KPM_FP32) {
        const int nz = (int)members[k].size();
        KPM_TRY(launch_cheb_step_batched(p, nz, bps[k], 0, 0, sk, maps_of[k]));
        for (int mm = 1; mm <= M - 2; ++mm) KPM_TRY(launch_cheb_step_batched(p, nz, bps[k], mm, 1, sk, maps_of[k]));
      } else {
        for (size_t z = 0; z < members[k].size(); ++z) {
          kpm_ctx::Cell& C = ctx->cells[members[k][z]];
          KPM_TRY(launch_cheb_step(p, prec, C.table, C.A, C.B, 0, C.acc, C.am, C.ao, 0, 0, sk));
          for (int mm = 1; mm <= M - 2; ++mm) {
            const void* cur = (mm & 1) ? C.B : C.A;
            void* out = (mm & 1) ? C.A : C.B;
            KPM_TRY(launch_cheb_step(p, prec, C.table, cur, out, 0, C.acc, C.am, C.ao, mm, 1, sk));
          }
        }
      }
      KPM_TRY(cudaEventRecord(ctx->fork_ev[k], sk));
      KPM_TRY(cudaStreamWaitEvent(c0, ctx->fork_ev[k], 0));
    }
    if (nitems > 0) {
      // every moment of every persistent cell in one launch, concurrent with
      // the per-step launches of the other shape classes
      KPM_TRY(cudaMemsetAsync(d_counter, 0, sizeof(int), c0));
      KPM_TRY(cudaEventRecordWithFlags(ctx->pev[0], c0, cudaEventRecordExternal));
      KPM_TRY(launch_cheb_persist(d_cells, d_items, nitems, d_counter, M, nclu, psmem, d_xbuf, nx_max, c0));
      KPM_TRY(cudaEventRecordWithFlags(ctx->pev[1], c0, cudaEventRecordExternal));
    }
    for (int c = 0; c < ncell; ++c) {
      kpm_ctx::Cell& C = ctx->cells[c];
      const int N = models[c].nx * models[c].ny;
      const ChebPlan& p = plans[C.cls];
      if (M >= 2 && !persist[C.cls])
        KPM_TRY(launch_cheb_gather(p, prec, ((M - 1) & 1) ? C.B : C.A, 0, C.acc, C.am, C.ao, M - 1, c0));
      KPM_TRY(launch_assemble(models[c].nx, models[c].ny, C.acc, C.misc, C.obs, C.misc + 3, ctx->bred, c0));
      KPM_TRY(launch_update(N, params[c], C.obs, mu_eff + c, ropts[c], C.misc + 4, ctx->bred, c0));
      KPM_TRY(cudaMemcpyAsync(ctx->bhost + 16 * c, C.misc, 8 * sizeof(double), cudaMemcpyDeviceToHost, c0));
    }
#undef KPM_TRY
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c0, &graph);
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(ctx, e, (std::string("capture of the batched iteration at ") + where).c_str());
    }
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->bgraph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->bgraph = nullptr;
      return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    ctx->bkey = key;
  }

  cudaStream_t s = (cudaStream_t)stream;
  std::vector<kpm_rmft_stats> st(ncell);
  memset(st.data(), 0, sizeof(kpm_rmft_stats) * ncell);
  int status = KPM_OK;
  double pms = 0.0;
  for (int it = 0; it < n_iter; ++it) {
    KPM_CU(cudaGraphLaunch(ctx->bgraph, s));
    KPM_CU(cudaStreamSynchronize(s));
    if (ctx->p_launched) {
      float ms = 0.f;
      KPM_CU(cudaEventElapsedTime(&ms, ctx->pev[0], ctx->pev[1]));
      pms += ms;
    }
    bool all = true;
    for (int c = 0; c < ncell; ++c) {
      const double* h = ctx->bhost + 16 * c;
      kpm_rmft_stats& q = st[c];
      q.a = h[0];
      q.b = h[1];
      q.mu = h[2];
      q.omega = h[3];
      q.residual = h[4];
      q.density_error = h[5];
      q.iterations = it + 1;
      if (!(q.residual == q.residual) || !(q.omega == q.omega) || q.residual > 1e300) {
        status = device_fault_status(ctx);
        if (status == KPM_OK) status = fail(ctx, KPM_ENONFINITE, "non-finite order parameters in a batched cell");
      }
      q.converged = q.residual < ropts[c].tol && fabs(q.density_error) < ropts[c].tol;
      all = all && q.converged;
    }
    if (status != KPM_OK || all) break;
  }
  // the persistent launch serves every cell: its time and streaming-equivalent
  // bytes are reported on each cell of the batch
  for (auto& q : st) {
    q.recursion_ms = pms;
    q.recursion_bytes = ctx->p_launched ? ctx->p_bytes * (double)(q.iterations) : 0.0;
    q.recursion_launches = ctx->p_launched ? 1 : 0;
  }
  if (stats) memcpy(stats, st.data(), sizeof(kpm_rmft_stats) * ncell);
  return status;
}


int kpm_autotune(kpm_ctx* ctx, const kpm_model* model, const kpm_opts* opts, const double* fields, const double* ab,
                 kpm_opts* best, double* best_ms_per_step, void* stream) {
  if (!ctx) return KPM_EINVAL;
  int r;
  if ((r = check_model(ctx, model))) return r;
  if ((r = check_dev(ctx, fields, "fields")) || (r = check_dev(ctx, ab, "ab"))) return r;
  if (!opts || !best) return fail(ctx, KPM_EINVAL, "null argument");
  DeviceGuard g(ctx->device);
  const int N = model->nx * model->ny;
  const int64_t D = 2 * (int64_t)N;
  const int prec = opts->precision;
  *best = *opts;
  auto key = std::make_tuple(model->nx, model->ny, prec, (opts->flags & KPM_FLAG_PH_HALF) ? 1 : 0, opts->probe_p,
                             opts->M);
  auto hit = ctx->tuned.find(key);
  if (hit != ctx->tuned.end()) {
    best->block_width = std::get<0>(hit->second);
    best->cols_per_block = std::get<1>(hit->second);
    best->flags = (opts->flags & ~KPM_FLAG_DOUBLE_STEP) | std::get<2>(hit->second);
    best->band_rows = std::get<3>(hit->second);
    if (best_ms_per_step) *best_ms_per_step = -1.0;
    return KPM_OK;
  }
  if ((r = ensure_site_scratch(ctx, N))) return r;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  KPM_CU(cudaEventCreate(&e0));
  KPM_CU(cudaEventCreate(&e1));
  // candidates: full width and narrower slabs (down to L2-resident ones), every column chunk
  // start vectors of a pass
  const int64_t ncols = opts->probe_p > 0 ? std::min<int64_t>(D, 2 * (int64_t)opts->probe_p * opts->probe_p)
                      : (opts->flags & KPM_FLAG_PH_HALF) ? D / 2 : D;
  std::vector<int64_t> widths = {ncols};
  for (int64_t w : {8192, 4096, 2048, 1024, 512, 384, 256, 128}) {
    const int64_t bw = balanced_width(ncols, w);
    if (bw < widths.back()) widths.push_back(bw);
  }
  std::vector<int> cols = prec == KPM_FP32 ? std::vector<int>{16, 8, 4} : std::vector<int>{8, 4, 2};
  // two trial orders: their difference is the per-moment time without the
  // per-slab start and gather, and the line through both predicts the pass
  // at the requested order (one wide slab has the least start/gather time, but
  // not always the fastest steps)
  const int Mt1 = 18, Mt2 = 34;
  const double Mreq = (double)std::max(opts->M, 2);
  double best_t = 1e300, best_step = 0.0;
  int best_w = 0, best_c = 0, best_f = 0, best_b = 0;
  std::vector<int> modes = prec == KPM_FP32 ? std::vector<int>{0, KPM_FLAG_DOUBLE_STEP} : std::vector<int>{0};
  for (int64_t w : widths) {
    for (int c : cols) for (int mode : modes) {
      kpm_opts o = *opts;
      o.M = Mt2;
      o.site_begin = o.site_end = 0;
      o.block_width = (int)w;
      o.cols_per_block = c;
      o.band_rows = 0;
      o.flags = (opts->flags & ~KPM_FLAG_DOUBLE_STEP) | mode;
      PassPlan pp;
      if (plan_pass(ctx, model, &o, &pp) != KPM_OK) continue;
      if (pp.cheb.cb != c) continue;  // chunk does not fit for this lattice
      if (mode && !pp.dbl) continue;  // no double-step plan for this lattice
      // band heights of the one-step kernels: the default (the wave model's
      // best), its next two, and one band per chunk (the double-step kernel
      // keeps its own bands)
      int bands[4] = {0, 0, 0, 0};
      int nband = 1;
      if (!mode) {
        int cand[4];
        int nc = band_rows_candidates(model->ny, pp.cheb.ldv / pp.cheb.cb, cand, 3);
        cand[nc++] = model->ny;
        for (int k = 0; k < nc; ++k) {
          bool seen = cand[k] == pp.cheb.ylen;
          for (int j = 1; j < nband; ++j) seen = seen || bands[j] == cand[k];
          if (!seen) bands[nband++] = cand[k];
        }
      }
      for (int bk = 0; bk < nband && !r; ++bk) {
        o.band_rows = bands[bk];
        o.M = Mt2;
        if (bk && plan_pass(ctx, model, &o, &pp) != KPM_OK) continue;
        if ((r = ensure_pass_scratch(ctx, model, &o, pp))) break;
        // one warm-up pass, then one timed pass at each trial order
        if ((r = enqueue_pass(ctx, model, &o, pp, fields, ab, ctx->obs, nullptr, s))) break;
        float ms[2] = {0.f, 0.f};
        for (int k = 0; k < 2 && !r; ++k) {
          o.M = k ? Mt2 : Mt1;
          KPM_CU(cudaEventRecord(e0, s));
          if ((r = enqueue_pass(ctx, model, &o, pp, fields, ab, ctx->obs, nullptr, s))) break;
          KPM_CU(cudaEventRecord(e1, s));
          KPM_CU(cudaEventSynchronize(e1));
          KPM_CU(cudaEventElapsedTime(&ms[k], e0, e1));
        }
        if (r) break;
        const double per_step = std::max(0.0, (double)(ms[1] - ms[0]) / (Mt2 - Mt1));
        const double predicted = ms[0] + per_step * (Mreq - Mt1);
        if (predicted < best_t) {
          best_t = predicted;
          best_step = per_step;
          best_w = o.block_width;
          best_c = c;
          best_f = mode;
          best_b = o.band_rows;
        }
      }
      if (r) break;
    }
    if (r) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r) return r;
  if (best_c == 0) return fail(ctx, KPM_EINVAL, "no recursion configuration fits this lattice");
  ctx->tuned[key] = std::make_tuple(best_w, best_c, best_f, best_b);
  best->block_width = best_w;
  best->band_rows = best_b;
  best->cols_per_block = best_c;
  best->flags = (opts->flags & ~KPM_FLAG_DOUBLE_STEP) | best_f;
  if (best_ms_per_step) *best_ms_per_step = best_step;
  return KPM_OK;
}

}  // extern "C"
