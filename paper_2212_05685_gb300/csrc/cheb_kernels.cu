// Block Chebyshev recursion of the KPM (App. B, Eq. alpha) on slabs of unit
// start vectors, as a fused complex stencil SpMM:
//
//   V_1 = h~ V_0,   V_{m+1} = 2 h~ V_m - V_{m-1},   V_0 = [e_{s0} ... e_{s0+b-1}]
//
// with the moment sums acc[J][s] += a_m V_m[K_s(J), J] over the nine local
// rows K_s(J) of every column (and the grand-potential series on the diagonal)
// fused into the step that reads V_m (Eqs. rho_KPM, F_KPM with unit r).
//
// Layout: V is row-major, V[K][c] with K = 2 i + alpha the Nambu row and c the
// column inside the slab; the row stride ldv is the slab width rounded up to
// the CTA's column chunk.  h~ is a 13-point stencil per row (diagonal, eight
// hops, four pairings), read from a per-site table of 2h~ entries.
//
// Each CTA owns a chunk of CB columns and a band of lattice rows y0..y1-1.  It
// marches along y keeping lattice rows y-1, y, y+1 of V_m (all Nx sites, both
// Nambu components, CB columns) in shared memory, with row y+2 and the next
// coefficient row in flight through cp.async, so every V_m element is read
// from global memory once per CTA while serving the 13 rows that need it.
// V_{m-1} is read and V_{m+1} written in place with coalesced 16-byte
// accesses.  No tensor cores: the stencil is sparse, not a dense contraction.
#include <algorithm>

#include "kpm_internal.cuh"

namespace kpm {
namespace {

// local rows of a unit column J = 2 j + beta (slot s): site j + (dx, dy),
// Nambu component beta, or 1 - beta for the pairing slots 5..8; slot 9
// repeats the diagonal for the grand-potential series.
__constant__ int kSlotDx[kSlots] = {0, 1, 0, 1, 1, 1, 0, -1, 0, 0};
__constant__ int kSlotDy[kSlots] = {0, 0, 1, 1, -1, 0, 1, 0, -1, 0};
__constant__ int kSlotFlip[kSlots] = {0, 0, 0, 0, 0, 1, 1, 1, 1, 0};

template <typename Real>
struct CT;
template <>
struct CT<float> {
  using C = float2;  // one complex
  using V = float4;  // VW complex values of a row
  static constexpr int VW = 2;
};
template <>
struct CT<double> {
  using C = double2;
  using V = double2;
  static constexpr int VW = 1;
};

__device__ __forceinline__ void cmac(float4& a, float2 c, float4 v) {
  a.x = fmaf(c.x, v.x, a.x);
  a.x = fmaf(-c.y, v.y, a.x);
  a.y = fmaf(c.x, v.y, a.y);
  a.y = fmaf(c.y, v.x, a.y);
  a.z = fmaf(c.x, v.z, a.z);
  a.z = fmaf(-c.y, v.w, a.z);
  a.w = fmaf(c.x, v.w, a.w);
  a.w = fmaf(c.y, v.z, a.w);
}
__device__ __forceinline__ void cmac(double2& a, double2 c, double2 v) {
  a.x = fma(c.x, v.x, a.x);
  a.x = fma(-c.y, v.y, a.x);
  a.y = fma(c.x, v.y, a.y);
  a.y = fma(c.y, v.x, a.y);
}
__device__ __forceinline__ void rmac(float4& a, float d, float4 v) {
  a.x = fmaf(d, v.x, a.x);
  a.y = fmaf(d, v.y, a.y);
  a.z = fmaf(d, v.z, a.z);
  a.w = fmaf(d, v.w, a.w);
}
__device__ __forceinline__ void rmac(double2& a, double d, double2 v) {
  a.x = fma(d, v.x, a.x);
  a.y = fma(d, v.y, a.y);
}
__device__ __forceinline__ float4 vneg(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }
__device__ __forceinline__ double2 vneg(double2 v) { return make_double2(-v.x, -v.y); }
__device__ __forceinline__ float4 vscale(float4 v, float s) { return make_float4(s * v.x, s * v.y, s * v.z, s * v.w); }
__device__ __forceinline__ double2 vscale(double2 v, double s) { return make_double2(s * v.x, s * v.y); }
template <typename V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <>
__device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// one lattice row of V (2 nx Nambu rows x CB columns) into shared memory
template <typename C, int CB>
__device__ __forceinline__ void stage_row(C* dst, const C* __restrict__ V, int ly, int nx, int64_t ldv,
                                          int64_t cb0) {
  constexpr int per_row = CB * (int)sizeof(C) / 16;
  const int total = 2 * nx * per_row;
  const C* base = V + (int64_t)(2 * nx) * ly * ldv + cb0;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int r = t / per_row, c = t - r * per_row;
    cp_async16(reinterpret_cast<char*>(dst + r * CB) + 16 * c,
               reinterpret_cast<const char*>(base + (int64_t)r * ldv) + 16 * c);
  }
}

// the 2h~ entries of one lattice row (nx sites x kCoef complex, contiguous)
template <typename C>
__device__ __forceinline__ void stage_coef(C* dst, const C* __restrict__ table, int ly, int nx) {
  const int chunks = nx * kCoef * (int)sizeof(C) / 16;
  const char* src = reinterpret_cast<const char*>(table + (int64_t)ly * nx * kCoef);
  char* d = reinterpret_cast<char*>(dst);
  for (int t = threadIdx.x; t < chunks; t += blockDim.x) cp_async16(d + 16 * t, src + 16 * t);
}

template <typename Real, int CB, int MODE>
__global__ void __launch_bounds__(512, 1)
    cheb_step_kernel(int nx, int ny, int64_t D, int64_t ldv, int ylen, const typename CT<Real>::C* __restrict__ table,
                     const typename CT<Real>::C* __restrict__ Vcur, typename CT<Real>::C* __restrict__ Vout,
                     int64_t s0, double2* __restrict__ acc, const double* __restrict__ am,
                     const double* __restrict__ ao, int m) {
  using C = typename CT<Real>::C;
  using V = typename CT<Real>::V;
  constexpr int VW = CT<Real>::VW;
  constexpr int NV = CB / VW;  // vectors per Nambu row of the chunk

  // shared memory: V_m window [4][2 nx][CB], V_{m-1} rows [2][2 nx][CB]
  // (step mode only), 2h~ rows [2][nx][kCoef]
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rowsz = 2 * nx * CB;
  C* win = reinterpret_cast<C*>(smem_raw);
  C* prev = win + 4 * rowsz;
  C* coef = prev + (MODE == 1 ? 2 * rowsz : 0);

  const int64_t cb0 = (int64_t)blockIdx.y * CB;
  const int y0 = blockIdx.x * ylen;
  const int y1 = min(ny, y0 + ylen);
  const int nrow = y1 - y0;

  // prologue: V_m rows y0-1, y0, y0+1, V_{m-1} row y0, coefficients of y0;
  // then V_m row y0+2, V_{m-1} row y0+1, coefficients of y0+1
  for (int q = 0; q < 3; ++q) stage_row<C, CB>(win + q * rowsz, Vcur, wrapi(y0 - 1 + q, ny), nx, ldv, cb0);
  if (MODE == 1) stage_row<C, CB>(prev, Vout, y0, nx, ldv, cb0);
  stage_coef<C>(coef, table, y0, nx);
  cp_commit();
  if (nrow >= 2) {
    stage_row<C, CB>(win + 3 * rowsz, Vcur, wrapi(y0 + 2, ny), nx, ldv, cb0);
    if (MODE == 1) stage_row<C, CB>(prev + rowsz, Vout, y0 + 1, nx, ldv, cb0);
    stage_coef<C>(coef + nx * kCoef, table, y0 + 1, nx);
  }
  cp_commit();

  const Real half = (Real)0.5;
  for (int q = 0; q < nrow; ++q) {
    const int y = y0 + q;
    cp_wait_1();
    __syncthreads();
    const C* wm = win + (q & 3) * rowsz;        // lattice row y - 1
    const C* w0 = win + ((q + 1) & 3) * rowsz;  // y
    const C* wp = win + ((q + 2) & 3) * rowsz;  // y + 1
    const C* pv = prev + (q & 1) * rowsz;       // V_{m-1}, row y
    const C* cf_row = coef + (q & 1) * nx * kCoef;

    for (int t = threadIdx.x; t < nx * NV; t += blockDim.x) {
      const int x = t / NV, v = t - x * NV;
      const int xr = x + 1 == nx ? 0 : x + 1;
      const int xl = x == 0 ? nx - 1 : x - 1;
      const int64_t K0 = 2 * ((int64_t)y * nx + x);
      const int64_t g0 = K0 * ldv + cb0 + v * VW;
#define KPM_LD(W, XX, AL) (*reinterpret_cast<const V*>((W) + (2 * (XX) + (AL)) * CB + v * VW))
      V a0, a1;
      if (MODE == 1) {
        a0 = vneg(KPM_LD(pv, x, 0));
        a1 = vneg(KPM_LD(pv, x, 1));
      } else {
        a0 = vzero<V>();
        a1 = vzero<V>();
      }
      const C* cf = cf_row + x * kCoef;
      {
        const C d = cf[0];
        rmac(a0, d.x, KPM_LD(w0, x, 0));
        rmac(a1, d.y, KPM_LD(w0, x, 1));
      }
      // neighbours k = 1..8: (+1,0) (-1,0) (0,+1) (0,-1) (+1,+1) (-1,-1) (+1,-1) (-1,+1)
      const C* wk[8] = {w0, w0, wp, wm, wp, wm, wm, wp};
      const int xk[8] = {xr, xl, x, x, xr, xl, xr, xl};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const V u0 = KPM_LD(wk[k], xk[k], 0);
        const V u1 = KPM_LD(wk[k], xk[k], 1);
        cmac(a0, cf[1 + k], u0);
        cmac(a1, cf[9 + k], u1);
        if (k < 4) {
          cmac(a0, cf[17 + k], u1);
          cmac(a1, cf[21 + k], u0);
        }
      }
#undef KPM_LD
      if (MODE == 0) {
        a0 = vscale(a0, half);
        a1 = vscale(a1, half);
      }
      *reinterpret_cast<V*>(Vout + g0) = a0;
      *reinterpret_cast<V*>(Vout + g0 + ldv) = a1;
    }

    if (MODE == 1) {
      // moment sums of the columns whose own site lies in lattice row y
      const double cm = am[m], co = ao[m];
      for (int t = threadIdx.x; t < CB * kSlots; t += blockDim.x) {
        const int c = t / kSlots, s = t - c * kSlots;
        const int64_t J = s0 + cb0 + c;
        if (J >= D) continue;
        const int64_t j = J >> 1;
        if (j / nx != y) continue;
        const int beta = (int)(J & 1);
        const int xs = wrapi((int)(j % nx) + kSlotDx[s], nx);
        const int dy = kSlotDy[s];
        const C* w = dy < 0 ? wm : (dy > 0 ? wp : w0);
        const int al = kSlotFlip[s] ? 1 - beta : beta;
        const C val = w[(2 * xs + al) * CB + c];
        const double coef_m = s == kSlots - 1 ? co : cm;
        double2* a = acc + J * kSlots + s;
        a->x += coef_m * (double)val.x;
        a->y += coef_m * (double)val.y;
      }
    }
    __syncthreads();
    // refill: V_m row y+3 into the buffer of y-1, V_{m-1} row y+2 and
    // coefficients of y+2 into the buffers of row y
    if (y + 3 <= y1) stage_row<C, CB>(win + (q & 3) * rowsz, Vcur, wrapi(y + 3, ny), nx, ldv, cb0);
    if (y + 2 < y1) {
      if (MODE == 1) stage_row<C, CB>(prev + (q & 1) * rowsz, Vout, y + 2, nx, ldv, cb0);
      stage_coef<C>(coef + (q & 1) * nx * kCoef, table, y + 2, nx);
    }
    cp_commit();
  }
  cp_wait_0();
}

// V0 = unit vectors e_{s0 + c} (zero elsewhere) and the m = 0 moment terms
template <typename C>
__global__ void cheb_init_kernel(int64_t D, int64_t ldv, C* __restrict__ V0, int64_t s0, double2* __restrict__ acc,
                                 const double* __restrict__ am, const double* __restrict__ ao) {
  const int64_t total = D * ldv;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t K = k / ldv, c = k - K * ldv;
    C v;
    v.x = K == s0 + c ? 1 : 0;
    v.y = 0;
    V0[k] = v;
  }
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ldv * kSlots;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = k / kSlots;
    const int s = (int)(k - c * kSlots);
    const int64_t J = s0 + c;
    if (J >= D) continue;
    double2 a = make_double2(0.0, 0.0);
    if (s == 0) a.x = am[0];
    if (s == kSlots - 1) a.x = ao[0];
    acc[J * kSlots + s] = a;
  }
}

// acc += a_m V[local rows] (the last moment, which no step reads again)
template <typename C>
__global__ void cheb_gather_kernel(int nx, int ny, int64_t D, int64_t ldv, int64_t width, const C* __restrict__ V,
                                   int64_t s0, double2* __restrict__ acc, const double* __restrict__ am,
                                   const double* __restrict__ ao, int m) {
  const int64_t total = width * kSlots;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = k / kSlots;
    const int s = (int)(k - c * kSlots);
    const int64_t J = s0 + c;
    if (J >= D) continue;
    const int64_t j = J >> 1;
    const int beta = (int)(J & 1);
    const int xs = wrapi((int)(j % nx) + kSlotDx[s], nx);
    const int ys = wrapi((int)(j / nx) + kSlotDy[s], ny);
    const int al = kSlotFlip[s] ? 1 - beta : beta;
    const int64_t K = 2 * ((int64_t)ys * nx + xs) + al;
    const C val = V[K * ldv + c];
    const double cf = s == kSlots - 1 ? ao[m] : am[m];
    double2* a = acc + J * kSlots + s;
    a->x += cf * (double)val.x;
    a->y += cf * (double)val.y;
  }
}

template <typename Real, int CB>
size_t smem_bytes(int nx) {  // step mode (the larger of the two)
  using C = typename CT<Real>::C;
  return sizeof(C) * ((size_t)6 * 2 * nx * CB + (size_t)2 * nx * kCoef);
}

template <typename Real, int CB, int MODE>
cudaError_t set_smem(int nx) {
  return cudaFuncSetAttribute(cheb_step_kernel<Real, CB, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes<Real, CB>(nx));
}

template <typename Real, int CB>
cudaError_t launch_step_t(const ChebPlan& p, const void* table, const void* Vcur, void* Vout, int64_t s0,
                          double2* acc, const double* am, const double* ao, int m, int mode, cudaStream_t s) {
  using C = typename CT<Real>::C;
  const dim3 grid((p.ny + p.ylen - 1) / p.ylen, (unsigned)(p.ldv / CB));
  if (mode == 0)
    cheb_step_kernel<Real, CB, 0><<<grid, p.nthreads, p.smem, s>>>(
        p.nx, p.ny, p.D, p.ldv, p.ylen, (const C*)table, (const C*)Vcur, (C*)Vout, s0, acc, am, ao, m);
  else
    cheb_step_kernel<Real, CB, 1><<<grid, p.nthreads, p.smem, s>>>(
        p.nx, p.ny, p.D, p.ldv, p.ylen, (const C*)table, (const C*)Vcur, (C*)Vout, s0, acc, am, ao, m);
  return cudaGetLastError();
}

constexpr size_t kSmemLimit = 227 * 1024;
constexpr int kSMs = 152;

}  // namespace

ChebPlan plan_cheb(int nx, int ny, int64_t width, int precision, int cb_request) {
  ChebPlan p;
  p.nx = nx;
  p.ny = ny;
  p.D = 2 * (int64_t)nx * ny;
  p.nthreads = 512;
  // widest chunk that fits shared memory (FP32: 16 columns, FP64: 8)
  int cands32[4] = {16, 8, 4, 2};
  int cands64[4] = {8, 4, 2, 1};
  int* c = precision == KPM_FP32 ? cands32 : cands64;
  p.cb = 0;
  const int min_cb = c[3];
  if (cb_request > 0 && cb_request < min_cb) cb_request = min_cb;
  for (int k = 0; k < 4; ++k) {
    if (cb_request > 0 && c[k] > cb_request) continue;
    const size_t sm = precision == KPM_FP32
                          ? (c[k] == 16 ? smem_bytes<float, 16>(nx)
                             : c[k] == 8 ? smem_bytes<float, 8>(nx)
                             : c[k] == 4 ? smem_bytes<float, 4>(nx)
                                         : smem_bytes<float, 2>(nx))
                          : (c[k] == 8 ? smem_bytes<double, 8>(nx)
                             : c[k] == 4 ? smem_bytes<double, 4>(nx)
                             : c[k] == 2 ? smem_bytes<double, 2>(nx)
                                         : smem_bytes<double, 1>(nx));
    if (sm <= kSmemLimit) {
      p.cb = c[k];
      p.smem = sm;
      break;
    }
  }
  if (p.cb == 0) {
    p.ldv = 0;
    return p;
  }
  p.ldv = (width + p.cb - 1) / p.cb * p.cb;
  // enough CTAs to fill the GPU a few times over: split y only when the
  // column chunks alone do not
  const int64_t chunks = p.ldv / p.cb;
  const int64_t want = 4 * kSMs;
  int yblocks = (int)std::min<int64_t>(ny, std::max<int64_t>(1, (want + chunks - 1) / chunks));
  p.ylen = std::max(1, (ny + yblocks - 1) / yblocks);
  return p;
}

cudaError_t cheb_prepare(const ChebPlan& p, int precision) {
  cudaError_t e = cudaSuccess;
  if (precision == KPM_FP32) {
    switch (p.cb) {
      case 16: if ((e = set_smem<float, 16, 0>(p.nx)) == cudaSuccess) e = set_smem<float, 16, 1>(p.nx); break;
      case 8: if ((e = set_smem<float, 8, 0>(p.nx)) == cudaSuccess) e = set_smem<float, 8, 1>(p.nx); break;
      case 4: if ((e = set_smem<float, 4, 0>(p.nx)) == cudaSuccess) e = set_smem<float, 4, 1>(p.nx); break;
      case 2: if ((e = set_smem<float, 2, 0>(p.nx)) == cudaSuccess) e = set_smem<float, 2, 1>(p.nx); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (p.cb) {
      case 8: if ((e = set_smem<double, 8, 0>(p.nx)) == cudaSuccess) e = set_smem<double, 8, 1>(p.nx); break;
      case 4: if ((e = set_smem<double, 4, 0>(p.nx)) == cudaSuccess) e = set_smem<double, 4, 1>(p.nx); break;
      case 2: if ((e = set_smem<double, 2, 0>(p.nx)) == cudaSuccess) e = set_smem<double, 2, 1>(p.nx); break;
      case 1: if ((e = set_smem<double, 1, 0>(p.nx)) == cudaSuccess) e = set_smem<double, 1, 1>(p.nx); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return e;
}

cudaError_t launch_cheb_init(const ChebPlan& p, int precision, void* V0, int64_t s0, double2* acc, const double* am,
                             const double* ao, cudaStream_t s) {
  const int64_t total = p.D * p.ldv;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 8 * kSMs * 4);
  if (precision == KPM_FP32)
    cheb_init_kernel<float2><<<grid, 256, 0, s>>>(p.D, p.ldv, (float2*)V0, s0, acc, am, ao);
  else
    cheb_init_kernel<double2><<<grid, 256, 0, s>>>(p.D, p.ldv, (double2*)V0, s0, acc, am, ao);
  return cudaGetLastError();
}

cudaError_t launch_cheb_step(const ChebPlan& p, int precision, const void* table, const void* Vcur, void* Vout,
                             int64_t s0, double2* acc, const double* am, const double* ao, int m, int mode,
                             cudaStream_t s) {
  if (precision == KPM_FP32) {
    switch (p.cb) {
      case 16: return launch_step_t<float, 16>(p, table, Vcur, Vout, s0, acc, am, ao, m, mode, s);
      case 8: return launch_step_t<float, 8>(p, table, Vcur, Vout, s0, acc, am, ao, m, mode, s);
      case 4: return launch_step_t<float, 4>(p, table, Vcur, Vout, s0, acc, am, ao, m, mode, s);
      case 2: return launch_step_t<float, 2>(p, table, Vcur, Vout, s0, acc, am, ao, m, mode, s);
    }
  } else {
    switch (p.cb) {
      case 8: return launch_step_t<double, 8>(p, table, Vcur, Vout, s0, acc, am, ao, m, mode, s);
      case 4: return launch_step_t<double, 4>(p, table, Vcur, Vout, s0, acc, am, ao, m, mode, s);
      case 2: return launch_step_t<double, 2>(p, table, Vcur, Vout, s0, acc, am, ao, m, mode, s);
      case 1: return launch_step_t<double, 1>(p, table, Vcur, Vout, s0, acc, am, ao, m, mode, s);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cheb_gather(const ChebPlan& p, int precision, const void* V, int64_t s0, double2* acc,
                               const double* am, const double* ao, int m, cudaStream_t s) {
  const int64_t width = p.ldv;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((width * kSlots + 255) / 256, 4 * kSMs));
  if (precision == KPM_FP32)
    cheb_gather_kernel<float2><<<grid, 256, 0, s>>>(p.nx, p.ny, p.D, p.ldv, width, (const float2*)V, s0, acc, am,
                                                    ao, m);
  else
    cheb_gather_kernel<double2><<<grid, 256, 0, s>>>(p.nx, p.ny, p.D, p.ldv, width, (const double2*)V, s0, acc,
                                                     am, ao, m);
  return cudaGetLastError();
}

}  // namespace kpm
