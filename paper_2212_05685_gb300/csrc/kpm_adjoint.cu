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
// accumulation of G (FP32 or FP64 products, FP64 per-warp partial sums without
// atomics) and the chain from G to the fields (eps, T, D).
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
                                    double g_omega, double2* __restrict__ w, int sb, int se) {
  const int N = nx * ny;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double* gn = g;
  const double* gc = g + 2 * N;
  const double* gF = g + 18 * N;
  double2* w0 = w + (size_t)(2 * j) * kSlots;
  double2* w1 = w + (size_t)(2 * j + 1) * kSlots;
  if (j < sb || j >= se) {  // columns outside the pass's site range
    for (int k = 0; k < kSlots; ++k) w0[k] = w1[k] = make_double2(0.0, 0.0);
    return;
  }
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

// Stencil-entry sums of the adjoint:
//   G[I][t] += coef * sum_{c in slab} lam[I, c] conj(alpha[K_t(I), c])
// for the 13 entries t of every row I (t = 0 the diagonal, 1..8 the hops to
// the same Nambu row of the neighbours (+1,0) (-1,0) (0,+1) (0,-1) (+1,+1)
// (-1,-1) (+1,-1) (-1,+1), 9..12 the pairings to the other Nambu row of the
// four nearest neighbours).  The slab's columns are dealt to `groups` sets;
// exactly one warp (FP64) or CTA (FP32) adds the set's sum for a given row
// to P[set][I][t], so the sums are deterministic (fixed order within a
// launch, launches in stream order); the sets are added in fixed order at
// the end (grad_reduce_kernel).
//
// FP64 slabs (interleaved complex): one warp owns one (row, set), its lanes
// stride over the set's columns with all 13 alpha rows loaded before the
// products, and lane t adds the warp's sum for entry t.  The FP64 path is
// bound by the FP64 pipe, not by these loads.
constexpr int kGradRows = 8;  // warps (rows) per CTA

__global__ void __launch_bounds__(kGradRows * 32, 2)
grad_rows_f64_kernel(int nx, int ny, int64_t ldv, const double2* __restrict__ lam,
                     const double2* __restrict__ alpha, double coef, double2* __restrict__ P) {
  const int64_t D = 2 * (int64_t)nx * ny;
  const int lane = threadIdx.x & 31;
  const int64_t R = (int64_t)blockIdx.x * kGradRows + (threadIdx.x >> 5);
  if (R >= D) return;  // uniform per warp; the kernel has no block barrier
  const int groups = gridDim.y;
  const int i = (int)(R >> 1), r = (int)(R & 1);
  const int x = i % nx, y = i / nx;
  const double2* rows[13];
  rows[0] = alpha + R * ldv;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t j = wrapi(x + kNbX[k], nx) + (int64_t)nx * wrapi(y + kNbY[k], ny);
    rows[1 + k] = alpha + (2 * j + r) * ldv;
    if (k < 4) rows[9 + k] = alpha + (2 * j + 1 - r) * ldv;
  }
  const double2* lrow = lam + R * ldv;
  double2 acc[13];
#pragma unroll
  for (int t = 0; t < 13; ++t) acc[t] = make_double2(0.0, 0.0);
  for (int64_t c = (int64_t)blockIdx.y * 32 + lane; c < ldv; c += (int64_t)groups * 32) {
    const double2 l = lrow[c];
    double2 v[13];
#pragma unroll
    for (int t = 0; t < 13; ++t) v[t] = rows[t][c];
#pragma unroll
    for (int t = 0; t < 13; ++t) {
      acc[t].x += l.x * v[t].x + l.y * v[t].y;
      acc[t].y += l.y * v[t].x - l.x * v[t].y;
    }
  }
  double2 mine = make_double2(0.0, 0.0);
#pragma unroll
  for (int t = 0; t < 13; ++t) {
    double re = acc[t].x, im = acc[t].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == t) mine = make_double2(re, im);
  }
  if (lane < 13) {
    double2* e = P + ((int64_t)blockIdx.y * D + R) * 13 + lane;
    e->x += coef * mine.x;
    e->y += coef * mine.y;
  }
}

// FP32 slabs: a tile of kTX x kTY sites per CTA, both Nambu rows, one lane per
// site.  Column pairs stream through shared memory kQ at a time (two stages
// in flight through cp.async): the alpha rows of the tile and its one-site
// halo (every alpha row is fetched once per tile instead of once per stencil
// entry) and the tile's own lambda rows.  Each lane keeps its 26 sums in FP32
// registers across every column pair its CTA visits, so no cross-lane
// reduction runs inside the loop; the two halves of the CTA take alternate
// pairs of a stage and are combined once at the end.  Column blocks are dealt
// to `groups` CTAs per tile; CTA (tile, set) is the only writer of
// P[set][rows of the tile][*].
constexpr int kTX = 16, kTY = 8, kQ = 8;
constexpr int kTileSites = kTX * kTY;                   // 128 lanes per half
constexpr int kHX = kTX + 2, kHY = kTY + 2;
constexpr int kSA = (kHX * kHY) | 1;                   // odd strides: conflict-free
constexpr int kSL = kTileSites | 1;                     //   16-byte shared accesses
constexpr int kStage = 2 * kQ * kSA + 2 * kQ * kSL;     // float4 per stage
constexpr size_t kTileSmem = 2 * kStage * sizeof(float4);
constexpr int kTileThreads = 2 * kTileSites;

__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_group1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_group0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Copy plan of one thread, the same for every stage: thread t copies pair
// q = t % kQ of the rows it owns (kQ divides the block size), so only the
// row and the shared-memory slot vary across its items.
constexpr int kAItems = (kHX * kHY * 2 * kQ + kTileThreads - 1) / kTileThreads;
constexpr int kLItems = (kTileSites * 2 * kQ) / kTileThreads;
static_assert(kTileThreads % kQ == 0 && (kTileSites * 2 * kQ) % kTileThreads == 0, "copy plan");

struct TileCopyPlan {
  int arow[kAItems], aslot[kAItems];  // alpha halo rows (arow < 0: no item)
  int lrow[kLItems], lslot[kLItems];  // lambda rows of the tile (lrow < 0: outside the lattice)
};

__device__ __forceinline__ void tile_copy_plan(TileCopyPlan& c, int nx, int ny, int x0, int y0) {
  const int q = threadIdx.x % kQ;
#pragma unroll
  for (int k = 0; k < kAItems; ++k) {
    const int it = threadIdx.x + k * kTileThreads;
    const int rn = it / kQ, n = rn & 1, h = rn >> 1;
    c.arow[k] = -1;
    c.aslot[k] = 0;
    if (it < kHX * kHY * 2 * kQ) {
      const int gx = wrapi(x0 - 1 + h % kHX, nx), gy = wrapi(y0 - 1 + h / kHX, ny);
      c.arow[k] = 2 * (gy * nx + gx) + n;
      c.aslot[k] = (n * kQ + q) * kSA + h;
    }
  }
#pragma unroll
  for (int k = 0; k < kLItems; ++k) {
    const int it = threadIdx.x + k * kTileThreads;
    const int rn = it / kQ, n = rn & 1, t = rn >> 1;
    const int sx = x0 + t % kTX, sy = y0 + t / kTX;
    c.lrow[k] = (sx < nx && sy < ny) ? 2 * (sy * nx + sx) + n : -1;
    c.lslot[k] = (n * kQ + q) * kSL + t;
  }
}

__device__ __forceinline__ void grad_tile_load(float4* stage, const TileCopyPlan& c, int64_t ldq, int64_t p0,
                                               const float4* __restrict__ lam, const float4* __restrict__ alpha) {
  float4* sa = stage;
  float4* sl = stage + 2 * kQ * kSA;
  const int64_t pq = p0 + threadIdx.x % kQ;
  const bool inq = pq < ldq;
  const int64_t pc = inq ? pq : 0;
#pragma unroll
  for (int k = 0; k < kAItems; ++k)
    if (c.arow[k] >= 0) cp_async16_zfill(sa + c.aslot[k], alpha + (int64_t)c.arow[k] * ldq + pc, inq ? 16 : 0);
#pragma unroll
  for (int k = 0; k < kLItems; ++k) {
    const bool ok = inq && c.lrow[k] >= 0;
    cp_async16_zfill(sl + c.lslot[k], lam + (ok ? (int64_t)c.lrow[k] * ldq + pc : 0), ok ? 16 : 0);
  }
  cp_commit_group();
}

__device__ __forceinline__ void pmac(float2& a, const float4& l, const float4& v) {
  a.x += l.x * v.x + l.z * v.z + l.y * v.y + l.w * v.w;
  a.y += l.z * v.x - l.x * v.z + l.w * v.y - l.y * v.w;
}

__global__ void __launch_bounds__(kTileThreads, 1)
grad_tile_f32_kernel(int nx, int ny, int64_t ldq, int tiles_x, const float4* __restrict__ lam,
                     const float4* __restrict__ alpha, double coef, double2* __restrict__ P) {
  extern __shared__ float4 gsm[];
  const int64_t D = 2 * (int64_t)nx * ny;
  const int x0 = (blockIdx.x % tiles_x) * kTX, y0 = (blockIdx.x / tiles_x) * kTY;
  const int groups = gridDim.y;
  const int64_t nblk = (ldq + kQ - 1) / kQ;
  const int half = threadIdx.x / kTileSites;
  const int ls = threadIdx.x % kTileSites;
  const int tx = ls % kTX, ty = ls / kTX;
  const bool valid = x0 + tx < nx && y0 + ty < ny;
  const int hc = (ty + 1) * kHX + tx + 1;
  float2 acc[26];
#pragma unroll
  for (int t = 0; t < 26; ++t) acc[t] = make_float2(0.f, 0.f);
  TileCopyPlan cp;
  tile_copy_plan(cp, nx, ny, x0, y0);

  int buf = 0;
  int64_t blk = blockIdx.y;
  if (blk < nblk) grad_tile_load(gsm, cp, ldq, blk * kQ, lam, alpha);
  for (; blk < nblk; blk += groups) {
    const int64_t nxt = blk + groups;
    if (nxt < nblk) {
      grad_tile_load(gsm + (buf ^ 1) * kStage, cp, ldq, nxt * kQ, lam, alpha);
      cp_wait_group1();
    } else {
      cp_wait_group0();
    }
    __syncthreads();
    if (valid) {
      const float4* sa = gsm + buf * kStage;
      const float4* sl = sa + 2 * kQ * kSA;
#pragma unroll 2
      for (int q = half; q < kQ; q += 2) {
        const float4* a0r = sa + q * kSA;          // Nambu row 0 of the halo at pair q
        const float4* a1r = sa + (kQ + q) * kSA;   // Nambu row 1
        const float4 l0 = sl[q * kSL + ls];
        const float4 l1 = sl[(kQ + q) * kSL + ls];
        pmac(acc[0], l0, a0r[hc]);
        pmac(acc[13], l1, a1r[hc]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int hk = hc + kNbY[k] * kHX + kNbX[k];
          const float4 b0 = a0r[hk], b1 = a1r[hk];
          pmac(acc[1 + k], l0, b0);
          pmac(acc[14 + k], l1, b1);
          if (k < 4) {
            pmac(acc[9 + k], l0, b1);
            pmac(acc[22 + k], l1, b0);
          }
        }
      }
    }
    __syncthreads();  // the next iteration's copies overwrite this stage
    buf ^= 1;
  }
  // combine the two halves (shared memory is free again) and add to P
  float2* red = reinterpret_cast<float2*>(gsm);
  if (half == 1) {
#pragma unroll
    for (int t = 0; t < 26; ++t) red[t * kTileSites + ls] = acc[t];
  }
  __syncthreads();
  if (half == 0 && valid) {
    const int64_t site = (int64_t)(y0 + ty) * nx + x0 + tx;
#pragma unroll
    for (int t = 0; t < 26; ++t) {
      const float2 o = red[t * kTileSites + ls];
      double2* e = P + ((int64_t)blockIdx.y * D + 2 * site + (t >= 13)) * 13 + (t % 13);
      e->x += coef * ((double)acc[t].x + (double)o.x);
      e->y += coef * ((double)acc[t].y + (double)o.y);
    }
  }
}

// G[I][t] = sum over the column sets of P[set][I][t], sets in fixed order
__global__ void grad_reduce_kernel(int64_t n, int groups, const double2* __restrict__ P, double2* __restrict__ G) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double2 s = P[e];
    for (int g = 1; g < groups; ++g) {
      const double2 v = P[(int64_t)g * n + e];
      s.x += v.x;
      s.y += v.y;
    }
    G[e] = s;
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

// out = 1 when a[0..n) equals b[0..n) and c[0..k) equals d[0..k) bit for bit
__global__ void differ_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                              const double* __restrict__ c, const double* __restrict__ d, int k,
                              int* __restrict__ differ) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + k; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = i < n ? a[i] : c[i - n], y = i < n ? b[i] : d[i - n];
    if (__double_as_longlong(x) != __double_as_longlong(y)) atomicOr(differ, 1);
  }
}
}  // namespace

cudaError_t launch_same_doubles(const double* a, const double* b, int64_t n, const double* c, const double* d, int k,
                                int* flag, int* host, int* same, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + k + 255) / 256, 4 * kSMs));
  differ_kernel<<<grid, 256, 0, s>>>(a, b, n, c, d, k, flag);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(host, flag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *same = *host == 0;
  return cudaSuccess;
}

cudaError_t launch_seed_weights(int nx, int ny, const double* grad_obs, const double* ab, double g_omega,
                                double2* w, cudaStream_t s, int sb, int se) {
  const int N = nx * ny;
  seed_weights_kernel<<<(N + 127) / 128, 128, 0, s>>>(nx, ny, grad_obs, ab, g_omega, w, sb, se < 0 ? N : se);
  return cudaGetLastError();
}

cudaError_t launch_seed_scatter(const ChebPlan& p, int prec, void* lam, int64_t s0, const double2* w,
                                const double* am, const double* ao, int m, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((p.ldv + 127) / 128, 4 * kSMs));
  seed_scatter_kernel<<<grid, 128, 0, s>>>(p.nx, p.ny, p.D, p.ldv, p.ldv, prec, lam, s0, w, am, ao, m);
  return cudaGetLastError();
}

int grad_groups(const ChebPlan& p, int prec) {
  if (prec == KPM_FP32) {
    // one CTA per SM (158 KB of stages): about two waves of (tile, set) CTAs
    const int64_t tiles = (int64_t)((p.nx + kTX - 1) / kTX) * ((p.ny + kTY - 1) / kTY);
    const int64_t nblk = (p.ldv / 2 + kQ - 1) / kQ;
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>((2 * kSMs) / tiles, nblk), 64));
  }
  // about two waves of 24 row-warps per SM, at least one 32-column stride per set
  const int64_t want = (2 * kSMs * 24 + p.D - 1) / std::max<int64_t>(p.D, 1);
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(want, (p.ldv + 31) / 32), 16));
}

cudaError_t launch_grad_accum(const ChebPlan& p, int prec, const void* lam, const void* alpha, double coef,
                              double2* P, cudaStream_t s) {
  const int groups = grad_groups(p, prec);
  if (prec == KPM_FP32) {
    // per-function attribute of the current device (cheap host call)
    cudaError_t e = cudaFuncSetAttribute(grad_tile_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTileSmem);
    if (e != cudaSuccess) return e;
    const int tiles_x = (p.nx + kTX - 1) / kTX;
    const dim3 grid((unsigned)(tiles_x * ((p.ny + kTY - 1) / kTY)), (unsigned)groups);
    grad_tile_f32_kernel<<<grid, kTileThreads, kTileSmem, s>>>(p.nx, p.ny, p.ldv / 2, tiles_x, (const float4*)lam,
                                                               (const float4*)alpha, coef, P);
    return cudaGetLastError();
  }
  const dim3 grid((unsigned)((p.D + kGradRows - 1) / kGradRows), (unsigned)groups);
  grad_rows_f64_kernel<<<grid, kGradRows * 32, 0, s>>>(p.nx, p.ny, p.ldv, (const double2*)lam,
                                                        (const double2*)alpha, coef, P);
  return cudaGetLastError();
}

cudaError_t launch_grad_reduce(int64_t D, int groups, const double2* P, double2* G, cudaStream_t s) {
  const int64_t n = D * 13;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * kSMs));
  grad_reduce_kernel<<<grid, 256, 0, s>>>(n, groups, P, G);
  return cudaGetLastError();
}

cudaError_t launch_grad_fields(int nx, int ny, const double2* G, const double* ab, double* out, cudaStream_t s) {
  const int N = nx * ny;
  grad_fields_kernel<<<(N + 127) / 128, 128, 0, s>>>(nx, ny, G, ab, out);
  return cudaGetLastError();
}

}  // namespace kpm
