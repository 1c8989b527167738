// kpm_observables_noalloc: the KPM pass of kpm_observables without any
// device allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: code that runs under a memory manager owning the whole
// device heap (a pre-sized arena of an inference server or a simulation
// framework that forbids allocations outside its pool), and code on a
// latency-critical path where cudaMalloc/cudaFree would implicitly
// synchronise the device.  Such a caller still passes its own inputs and
// outputs; every intermediate (Chebyshev coefficients, the rescaled stencil
// table, the moment accumulators and the two recursion slabs) lives in the
// file-scope device array below instead of in a context's heap scratch.
//
// The array is part of the loaded module: every GPU that loads this library
// holds kNoAllocScratchBytes of it until the process exits.  Its device
// address is resolved with that device current (cudaGetSymbolAddress) by
// every call made outside stream capture, so a module reloaded after a
// context teardown (cudaDeviceReset) is found at its new address; a call made
// while its stream captures reuses the address of the last call outside
// capture on that device, so make one call before capturing.  Every call on a
// device shares the one array, so calls
// whose work overlaps on the GPU (different streams, or host threads racing)
// corrupt each other's intermediates: serialise them.  Each call writes every
// scratch byte it later reads, so nothing has to start at zero and a call
// never sees the previous call's contents.
#include <algorithm>
#include <mutex>

#include "kpm_internal.cuh"

namespace kpm {
namespace {

constexpr size_t kNoAllocScratchBytes = 48ull << 20;  // 48 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// device address of g_noalloc_scratch on `device` (current): resolved afresh
// unless `stream` is capturing, then the address of the last call outside
// capture (cudaErrorNotReady when there was none)
cudaError_t scratch_address(int device, cudaStream_t stream, void** out) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  if (!g_scratch_addr[device]) return cudaErrorNotReady;
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// device memory of GPU `dev` (or managed memory)
bool is_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace kpm

using namespace kpm;

extern "C" int kpm_observables_noalloc(const kpm_model* m, const kpm_opts* o, const double* fields,
                                       const double* ab, double* obs, double* omega, void* stream) {
  if (!m || !o || !fields || !ab || !obs) return KPM_EINVAL;
  if (m->nx < 2 || m->ny < 2 || o->M < 1) return KPM_EINVAL;
  if (o->precision != KPM_FP32 && o->precision != KPM_FP64) return KPM_EINVAL;
  if ((o->flags & KPM_FLAG_PH_HALF) || o->probe_p) return KPM_EINVAL;  // the exact full pass only
  if (o->block_width < 0 || o->cols_per_block < 0 || o->band_rows < 0) return KPM_EINVAL;
  if (o->site_begin != 0 || o->site_end != 0) return KPM_EINVAL;      // all sites
  if (!(o->temperature >= 0.0 && o->temperature < 1e300)) return KPM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return KPM_ECUDA;
  }
  if (!is_device(fields, dev) || !is_device(ab, dev) || !is_device(obs, dev) || (omega && !is_device(omega, dev)))
    return KPM_EINVAL;
  const int N = m->nx * m->ny;
  const int64_t D = 2 * (int64_t)N;
  const size_t elem = o->precision == KPM_FP32 ? 8 : 16;

  // fixed part of the layout: coefficients, reduction partials, stencil table, accumulators
  const size_t off_am = 0;
  const size_t off_ao = align256(off_am + (size_t)o->M * sizeof(double));
  const size_t off_red = align256(off_ao + (size_t)o->M * sizeof(double));
  const size_t off_tab = align256(off_red + (size_t)reduce_scratch_doubles(0) * sizeof(double));
  const size_t off_acc = align256(off_tab + (size_t)N * table_bytes_per_site(o->precision));
  const size_t off_slab = align256(off_acc + (size_t)D * kSlots * sizeof(double2));
  if (off_slab >= kNoAllocScratchBytes) return KPM_EINVAL;  // the lattice or M exceeds the static scratch

  // widest slab (unit columns per recursion) whose two buffers fit the rest
  const size_t avail = kNoAllocScratchBytes - off_slab;
  int64_t width = std::min<int64_t>(o->block_width > 0 ? o->block_width : D,
                                    (int64_t)(avail / (2 * (size_t)D * elem)));
  ChebPlan p;
  p.cb = 0;
  while (width >= 1) {
    p = plan_cheb(m->nx, m->ny, width, o->precision, o->cols_per_block, o->band_rows);
    if (p.cb == 0) return KPM_EINVAL;
    if (2 * (size_t)D * p.ldv * elem + 2 * 255 <= avail) break;
    width -= p.cb;
  }
  if (width < 1 || p.cb == 0) return KPM_EINVAL;  // not even one column chunk fits

  void* base = nullptr;
  cudaError_t e = scratch_address(dev, (cudaStream_t)stream, &base);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return KPM_ECUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  double* am = reinterpret_cast<double*>(b + off_am);
  double* ao = reinterpret_cast<double*>(b + off_ao);
  double* red = reinterpret_cast<double*>(b + off_red);
  void* table = b + off_tab;
  double2* acc = reinterpret_cast<double2*>(b + off_acc);
  void* A = b + off_slab;
  void* B = b + align256(off_slab + (size_t)D * p.ldv * elem);

  cudaStream_t s = (cudaStream_t)stream;
  const int M = o->M;
  const int prec = o->precision;
#define KPM_NA(expr)                 \
  do {                               \
    if ((expr) != cudaSuccess) {     \
      cudaGetLastError();            \
      return KPM_ECUDA;              \
    }                                \
  } while (0)
  KPM_NA(cheb_prepare(p, prec));
  KPM_NA(launch_coefficients(M, ab, am, ao, s, 0, o->temperature));
  if (prec == KPM_FP32)
    KPM_NA(launch_scale_table_f32(*m, fields, ab, (float2*)table, s));
  else
    KPM_NA(launch_scale_table_f64(*m, fields, ab, (double2*)table, s));
  for (int64_t s0 = 0; s0 < D; s0 += p.ldv) {  // padded width: each column in one slab
    KPM_NA(launch_cheb_init(p, prec, A, s0, acc, am, ao, s));
    if (M >= 2) KPM_NA(launch_cheb_step(p, prec, table, A, B, s0, acc, am, ao, 0, 0, s));
    for (int mm = 1; mm <= M - 2; ++mm) {
      const void* cur = (mm & 1) ? B : A;
      void* out = (mm & 1) ? A : B;
      KPM_NA(launch_cheb_step(p, prec, table, cur, out, s0, acc, am, ao, mm, 1, s));
    }
    if (M >= 2) KPM_NA(launch_cheb_gather(p, prec, ((M - 1) & 1) ? B : A, s0, acc, am, ao, M - 1, s));
  }
  KPM_NA(launch_assemble(m->nx, m->ny, acc, ab, obs, omega, red, s));
#undef KPM_NA
  return KPM_OK;
}
