// Adjoint of the KPM pass (App. B, Eqs. dFdH, dalphadH): kernels of the
// backward recursion.  For each unit column J the loss L = Re sum_m c_m^dag
// alpha_m, c_m = a_m w_J + a g_Omega a^Omega_m e_J, is differentiated by
//
//   lambda_m = c_m + 2 h~ lambda_{m+1} - lambda_{m+2},   m = M-1 .. 1,
//   G_IK    += lambda_1,I conj(alpha_0,K) + 2 sum_{m>=2} lambda_m,I conj(alpha_{m-1},K)
//
// over the 13 stencil entries (I, K) of every row (h~ is Hermitian, so the
// lambda recursion is the forward stencil SpMM).  The lambda steps reuse the
// recursion kernel; this file holds the seed scatter, the stencil-entry
// accumulation of G (FP64, one atomic per entry and CTA after a warp
// reduction) and the chain from G to the fields (eps, T, D).
#include <algorithm>

#include "kpm_internal.cuh"

namespace kpm {
namespace {

constexpr int kSMs = 152;

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// local rows of unit column J (same slots as the forward moment sums)
__constant__ int kSlotDx[kSlots] = {0, 1, 0, 1, 1, 1, 0, -1, 0, 0};
__constant__ int kSlotDy[kSlots] = {0, 0, 1, 1, -1, 0, 1, 0, -1, 0};
__constant__ int kSlotFlip[kSlots] = {0, 0, 0, 0, 0, 1, 1, 1, 1, 0};

// stencil neighbours k = 1..8 (hops) and nn k = 1..4 (pairings)
__constant__ int kNbX[8] = {1, -1, 0, 0, 1, -1, 1, -1};
__constant__ int kNbY[8] = {0, 0, 1, -1, 1, -1, -1, 1};

// element (K, c) of a slab, any precision/layout
__device__ __forceinline__ double2 slab_elem(const void* V, int prec, int64_t ldv, int64_t K, int64_t c) {
  if (prec == KPM_FP32) {
    const float4 q = reinterpret_cast<const float4*>(V)[K * (ldv / 2) + (c >> 1)];
    return (c & 1) ? make_double2(q.y, q.w) : make_double2(q.x, q.z);
  }
  return reinterpret_cast<const double2*>(V)[K * ldv + c];
}
__device__ __forceinline__ void slab_add(void* V, int prec, int64_t ldv, int64_t K, int64_t c, double re, double im) {
  if (prec == KPM_FP32) {
    float* q = reinterpret_cast<float*>(reinterpret_cast<float4*>(V) + K * (ldv / 2) + (c >> 1));
    q[c & 1] += (float)re;
    q[2 + (c & 1)] += (float)im;
  } else {
    double2* q = reinterpret_cast<double2*>(V) + K * ldv + c;
    q->x += re;
    q->y += im;
  }
}

// Seed weights of every unit column from the upstream gradients (readings
// N2, N3 transposed): w[J][s] with dL = Re sum conj(W_KJ) dF_KJ.
__global__ void seed_weights_kernel(int nx, int ny, const double* __restrict__ g, const double* __restrict__ ab,
                                    double g_omega, double2* __restrict__ w) {
  const int N = nx * ny;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double* gn = g;
  const double* gc = g + 2 * N;
  const double* gF = g + 18 * N;
  double2* w0 = w + (size_t)(2 * j) * kSlots;
  double2* w1 = w + (size_t)(2 * j + 1) * kSlots;
  w0[0] = make_double2(gn[j], 0.0);
  w1[0] = make_double2(-gn[N + j], 0.0);
  for (int d = 0; d < 4; ++d) {
    const double* c0 = gc + 2 * ((0 * 4 + d) * N + j);
    const double* c1 = gc + 2 * ((1 * 4 + d) * N + j);
    w0[1 + d] = make_double2(c0[0], c0[1]);    // chi_up = entry
    w1[1 + d] = make_double2(-c1[0], c1[1]);   // chi_dn = -conj(entry)
  }
  for (int e = 0; e < 4; ++e) {
    const double* f = gF + 2 * (e * N + j);
    w0[5 + e] = make_double2(-f[0], f[1]);     // F = -conj(entry)
    w1[5 + e] = make_double2(0.0, 0.0);
  }
  const double om = ab[0] * g_omega;           // Omega = a tr G_M(h~)
  w0[9] = make_double2(om, 0.0);
  w1[9] = make_double2(om, 0.0);
}

// lambda[K_s(J), c] += coef_s w[J][s] for the slab's columns, one thread per
// column (slots of one column may share a row on tiny tori)
__global__ void seed_scatter_kernel(int nx, int ny, int64_t D, int64_t ldv, int64_t width, int prec, void* lam,
                                    int64_t s0, const double2* __restrict__ w, const double* __restrict__ am,
                                    const double* __restrict__ ao, int m) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < width; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t J = s0 + c;
    if (J >= D) continue;
    const int64_t j = J >> 1;
    const int beta = (int)(J & 1);
    const double cm = am[m], co = ao[m];
    for (int s = 0; s < kSlots; ++s) {
      const double2 ws = w[J * kSlots + s];
      if (ws.x == 0.0 && ws.y == 0.0) continue;
      const int xs = wrapi((int)(j % nx) + kSlotDx[s], nx);
      const int ys = wrapi((int)(j / nx) + kSlotDy[s], ny);
      const int al = kSlotFlip[s] ? 1 - beta : beta;
      const int64_t K = 2 * ((int64_t)ys * nx + xs) + al;
      const double cf = s == kSlots - 1 ? co : cm;
      slab_add(lam, prec, ldv, K, c, cf * ws.x, cf * ws.y);
    }
  }
}

// G[I][k] += coef * sum_{c in slab} lam[I, c] conj(alpha[K_k(I), c]) for the
// 13 stencil entries of both Nambu rows of every site.  One warp per site
// and 32 columns: the products are reduced across the warp by shuffles, then
// one FP64 atomic per entry and warp.
constexpr int kGradCols = 32;  // columns per block
constexpr int kGradSites = 8;  // sites per block

__global__ void grad_accum_kernel(int nx, int ny, int64_t ldv, int prec, const void* __restrict__ lam,
                                  const void* __restrict__ alpha, double coef, double2* __restrict__ G) {
  const int N = nx * ny;
  const int tc = threadIdx.x % kGradCols;
  const int ts = threadIdx.x / kGradCols;
  const int i = blockIdx.x * kGradSites + ts;
  const int64_t c = (int64_t)blockIdx.y * kGradCols + tc;
  double2 acc[26];
#pragma unroll
  for (int k = 0; k < 26; ++k) acc[k] = make_double2(0.0, 0.0);
  if (i < N && c < ldv) {
    const int x = i % nx, y = i / nx;
    const double2 l0 = slab_elem(lam, prec, ldv, 2 * (int64_t)i, c);
    const double2 l1 = slab_elem(lam, prec, ldv, 2 * (int64_t)i + 1, c);
    // diagonal
    {
      const double2 a0 = slab_elem(alpha, prec, ldv, 2 * (int64_t)i, c);
      const double2 a1 = slab_elem(alpha, prec, ldv, 2 * (int64_t)i + 1, c);
      acc[0] = make_double2(l0.x * a0.x + l0.y * a0.y, l0.y * a0.x - l0.x * a0.y);
      acc[13] = make_double2(l1.x * a1.x + l1.y * a1.y, l1.y * a1.x - l1.x * a1.y);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int j = wrapi(x + kNbX[k], nx) + nx * wrapi(y + kNbY[k], ny);
      const double2 a0 = slab_elem(alpha, prec, ldv, 2 * (int64_t)j, c);
      const double2 a1 = slab_elem(alpha, prec, ldv, 2 * (int64_t)j + 1, c);
      // hops: (i,0)->(j,0), (i,1)->(j,1)
      acc[1 + k] = make_double2(l0.x * a0.x + l0.y * a0.y, l0.y * a0.x - l0.x * a0.y);
      acc[14 + k] = make_double2(l1.x * a1.x + l1.y * a1.y, l1.y * a1.x - l1.x * a1.y);
      if (k < 4) {  // pairings: (i,0)->(j,1), (i,1)->(j,0)
        acc[9 + k] = make_double2(l0.x * a1.x + l0.y * a1.y, l0.y * a1.x - l0.x * a1.y);
        acc[22 + k] = make_double2(l1.x * a0.x + l1.y * a0.y, l1.y * a0.x - l1.x * a0.y);
      }
    }
  }
  // reduce over the 32 columns of this site (one warp = one site)
#pragma unroll
  for (int k = 0; k < 26; ++k) {
    double re = acc[k].x, im = acc[k].y;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (tc == 0 && i < N && (re != 0.0 || im != 0.0)) {
      double2* g = G + (size_t)(2 * i + (k >= 13)) * 13 + (k % 13);
      atomicAdd(&g->x, coef * re);
      atomicAdd(&g->y, coef * im);
    }
  }
}

// FP32 slabs: the same sums with the products and the warp reduction in FP32
// (64 columns per warp, two per lane) and FP64 atomics, so the FP64 pipe
// (1/64 of the FP32 rate on this part) is used only for the final adds.
__device__ __forceinline__ float2 pconj2(float4 l, float4 a) {
  // sum over the pair of columns of l_c conj(a_c); layout (re0, re1, im0, im1)
  return make_float2(l.x * a.x + l.z * a.z + l.y * a.y + l.w * a.w,
                     l.z * a.x - l.x * a.z + l.w * a.y - l.y * a.w);
}

__global__ void grad_accum_f32_kernel(int nx, int ny, int64_t ldv, const float4* __restrict__ lam,
                                      const float4* __restrict__ alpha, double coef, double2* __restrict__ G) {
  const int N = nx * ny;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t ldq = ldv / 2;
  float2 acc[26];
#pragma unroll
  for (int k = 0; k < 26; ++k) acc[k] = make_float2(0.f, 0.f);
  if (i < N) {
    const int x = i % nx, y = i / nx;
    int64_t nb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) nb[k] = 2 * (int64_t)(wrapi(x + kNbX[k], nx) + nx * wrapi(y + kNbY[k], ny)) * ldq;
    const int64_t r0 = 2 * (int64_t)i * ldq;
    // each lane sums its column pairs over the whole slab in FP32 registers
    for (int64_t q = (int64_t)blockIdx.y * 32 + lane; q < ldq; q += (int64_t)gridDim.y * 32) {
      const float4 l0 = lam[r0 + q];
      const float4 l1 = lam[r0 + ldq + q];
      const float2 d0 = pconj2(l0, alpha[r0 + q]);
      const float2 d1 = pconj2(l1, alpha[r0 + ldq + q]);
      acc[0].x += d0.x;
      acc[0].y += d0.y;
      acc[13].x += d1.x;
      acc[13].y += d1.y;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 a0 = alpha[nb[k] + q];
        const float4 a1 = alpha[nb[k] + ldq + q];
        const float2 h0 = pconj2(l0, a0), h1 = pconj2(l1, a1);
        acc[1 + k].x += h0.x;
        acc[1 + k].y += h0.y;
        acc[14 + k].x += h1.x;
        acc[14 + k].y += h1.y;
        if (k < 4) {
          const float2 p0 = pconj2(l0, a1), p1 = pconj2(l1, a0);
          acc[9 + k].x += p0.x;
          acc[9 + k].y += p0.y;
          acc[22 + k].x += p1.x;
          acc[22 + k].y += p1.y;
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 26; ++k) {
    float re = acc[k].x, im = acc[k].y;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0 && i < N && (re != 0.f || im != 0.f)) {
      double2* g = G + (size_t)(2 * i + (k >= 13)) * 13 + (k % 13);
      atomicAdd(&g->x, coef * (double)re);
      atomicAdd(&g->y, coef * (double)im);
    }
  }
}

// dL/d(eps, T, D) from G (gradient in h~), divided by a (h~ = (h - b)/a).
//   stencil slots of row I: 0 diag, 1..8 hops to (+1,0) (-1,0) (0,+1) (0,-1)
//   (+1,+1) (-1,-1) (+1,-1) (-1,+1), 9..12 pairings to (+1,0) (-1,0) (0,+1) (0,-1)
__constant__ int kFwdSlot[4] = {1, 3, 5, 7};   // forward bond d -> hop slot at i
__constant__ int kBwdSlot[4] = {2, 4, 6, 8};   // the same bond seen from i + d
__constant__ int kPairSlot[4] = {9, 11, 10, 12};  // nn e = +x, +y, -x, -y -> pairing slot
__constant__ int kFwdDX[4] = {1, 0, 1, 1};
__constant__ int kFwdDY[4] = {0, 1, 1, -1};
__constant__ int kNnDX[4] = {1, 0, -1, 0};
__constant__ int kNnDY[4] = {0, 1, 0, -1};

__global__ void grad_fields_kernel(int nx, int ny, const double2* __restrict__ G, const double* __restrict__ ab,
                                   double* __restrict__ out) {
  const int N = nx * ny;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int x = i % nx, y = i / nx;
  const double ia = 1.0 / ab[0];
  const double2* g0 = G + (size_t)(2 * i) * 13;
  const double2* g1 = G + (size_t)(2 * i + 1) * 13;
  out[i] = g0[0].x * ia;
  out[N + i] = -g1[0].x * ia;
  for (int d = 0; d < 4; ++d) {
    const int j = wrapi(x + kFwdDX[d], nx) + nx * wrapi(y + kFwdDY[d], ny);
    const double2 f0 = g0[kFwdSlot[d]], b0 = G[(size_t)(2 * j) * 13 + kBwdSlot[d]];
    const double2 f1 = g1[kFwdSlot[d]], b1 = G[(size_t)(2 * j + 1) * 13 + kBwdSlot[d]];
    double* t0 = out + 2 * N + 2 * ((0 * 4 + d) * N + i);
    double* t1 = out + 2 * N + 2 * ((1 * 4 + d) * N + i);
    // T_up: G[(i0),(j0)] + conj(G[(j0),(i0)]);  T_dn: -(conj(G[(i1),(j1)]) + G[(j1),(i1)])
    t0[0] = (f0.x + b0.x) * ia;
    t0[1] = (f0.y - b0.y) * ia;
    t1[0] = -(f1.x + b1.x) * ia;
    t1[1] = -(-f1.y + b1.y) * ia;
  }
  for (int e = 0; e < 4; ++e) {
    const int j = wrapi(x + kNnDX[e], nx) + nx * wrapi(y + kNnDY[e], ny);
    const double2 f = g0[kPairSlot[e]];
    const double2 r = G[(size_t)(2 * j + 1) * 13 + kPairSlot[(e + 2) & 3]];
    double* q = out + 18 * N + 2 * (e * N + i);
    // D: -(G[(i0),(j1)] + conj(G[(j1),(i0)]))
    q[0] = -(f.x + r.x) * ia;
    q[1] = -(f.y - r.y) * ia;
  }
}

}  // namespace

cudaError_t launch_seed_weights(int nx, int ny, const double* grad_obs, const double* ab, double g_omega,
                                double2* w, cudaStream_t s) {
  const int N = nx * ny;
  seed_weights_kernel<<<(N + 127) / 128, 128, 0, s>>>(nx, ny, grad_obs, ab, g_omega, w);
  return cudaGetLastError();
}

cudaError_t launch_seed_scatter(const ChebPlan& p, int prec, void* lam, int64_t s0, const double2* w,
                                const double* am, const double* ao, int m, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((p.ldv + 127) / 128, 4 * kSMs));
  seed_scatter_kernel<<<grid, 128, 0, s>>>(p.nx, p.ny, p.D, p.ldv, p.ldv, prec, lam, s0, w, am, ao, m);
  return cudaGetLastError();
}

cudaError_t launch_grad_accum(const ChebPlan& p, int prec, const void* lam, const void* alpha, double coef,
                              double2* G, cudaStream_t s) {
  const int N = p.nx * p.ny;
  if (prec == KPM_FP32) {
    // a few column groups per site: enough CTAs for the GPU, few atomics per entry
    const int64_t groups = (p.ldv / 2 + 31) / 32;
    const int gy = (int)std::max<int64_t>(1, std::min<int64_t>(groups, std::max<int64_t>(1, 8 * 152 * 8 / std::max(N, 1))));
    const dim3 grid((N + 7) / 8, (unsigned)gy);
    grad_accum_f32_kernel<<<grid, 256, 0, s>>>(p.nx, p.ny, p.ldv, (const float4*)lam, (const float4*)alpha, coef, G);
    return cudaGetLastError();
  }
  const dim3 grid((N + kGradSites - 1) / kGradSites, (unsigned)((p.ldv + kGradCols - 1) / kGradCols));
  grad_accum_kernel<<<grid, kGradSites * kGradCols, 0, s>>>(p.nx, p.ny, p.ldv, prec, lam, alpha, coef, G);
  return cudaGetLastError();
}

cudaError_t launch_grad_fields(int nx, int ny, const double2* G, const double* ab, double* out, cudaStream_t s) {
  const int N = nx * ny;
  grad_fields_kernel<<<(N + 127) / 128, 128, 0, s>>>(nx, ny, G, ab, out);
  return cudaGetLastError();
}

}  // namespace kpm
