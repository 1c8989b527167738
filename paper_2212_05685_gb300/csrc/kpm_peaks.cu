// Measured ALU peaks of the device: the denominators of the rooflines of the
// FP64 recursion and of the double-float recursion (which runs on the FP32
// pipes).  Each thread advances 8 independent FMA chains, so the pipes see no
// dependent-issue stalls; 4 CTAs of 256 threads per SM.  Thread 0 of every CTA
// records %clock64 and %globaltimer around its loop for the SM clock.
#include <string.h>

#include <algorithm>
#include <vector>

#include "kpm_internal.cuh"

namespace kpm {
namespace {

constexpr int kChains = 8;

__device__ __forceinline__ double fma_rn(double x, double a, double b) { return __fma_rn(x, a, b); }
__device__ __forceinline__ float fma_rn(float x, float a, float b) { return __fmaf_rn(x, a, b); }

__device__ __forceinline__ void clock_stamp(unsigned long long* t) {
  unsigned long long c, g;
  asm volatile("mov.u64 %0, %%clock64;" : "=l"(c));
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g));
  t[0] = c;
  t[1] = g;
}

// SPREAD: each chain has its own multiplier and addend registers; else all
// chains share one pair (the two operand patterns favour different pipes'
// register-bank access, so the probe keeps the better of the two)
template <typename T, bool SPREAD>
__global__ void __launch_bounds__(256) fma_chain_kernel(int iters, T a, T b, T* sink, unsigned long long* clk) {
  __shared__ unsigned long long t0[2];
  if (threadIdx.x == 0) clock_stamp(t0);
  T x[kChains], y[kChains], z[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    x[k] = (T)(threadIdx.x + k);
    y[k] = SPREAD ? a + (T)k * (T)1e-9 : a;
    z[k] = SPREAD ? b * (T)(k + 1) : b;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = SPREAD ? fma_rn(x[k], y[k], z[k]) : fma_rn(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == (T)-1.2345) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the chains
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t1[2];
    clock_stamp(t1);
    clk[2 * blockIdx.x] = t1[0] - t0[0];
    clk[2 * blockIdx.x + 1] = t1[1] - t0[1];
  }
}

// packed pair of FP32 FMAs per instruction (fma.rn.f32x2)
__global__ void __launch_bounds__(256) fma_chain_f32x2_kernel(int iters, unsigned long long a, unsigned long long b,
                                                              float* sink, unsigned long long* clk) {
  __shared__ unsigned long long t0[2];
  if (threadIdx.x == 0) clock_stamp(t0);
  unsigned long long x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    const float v = (float)(threadIdx.x + k);
    asm("mov.b64 %0, {%1, %1};" : "=l"(x[k]) : "f"(v));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(a), "l"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
    s += lo + hi;
  }
  if (s == -1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t1[2];
    clock_stamp(t1);
    clk[2 * blockIdx.x] = t1[0] - t0[0];
    clk[2 * blockIdx.x + 1] = t1[1] - t0[1];
  }
}

unsigned long long pack2(float v) {
  unsigned int u;
  memcpy(&u, &v, 4);
  return ((unsigned long long)u << 32) | u;
}

}  // namespace

// out[0] FP64 TFLOP/s, out[1] FP32 TFLOP/s, out[2] f32x2 TFLOP/s, out[3] SM MHz;
// scratch: device, at least peak_scratch_bytes()
size_t peak_scratch_bytes(int sms) { return (size_t)sms * 4 * 256 * sizeof(double) + (size_t)sms * 4 * 16; }

cudaError_t measure_alu_peaks(int sms, void* scratch, double* out, cudaStream_t s) {
  const int grid = 4 * sms, threads = 256;
  double* sink = static_cast<double*>(scratch);
  unsigned long long* clk = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) +
                                                                   (size_t)grid * threads * sizeof(double));
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  const double threads_total = (double)grid * threads;
  double best[3] = {0.0, 0.0, 0.0};
  double mhz = 0.0;
  std::vector<unsigned long long> hclk(2 * (size_t)grid);
  for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
    // flops per thread-iteration: 8 chains x 2 (x 2 packed)
    const int iters = kind == 0 ? 2048 : (kind == 1 ? 65536 : 32768);
    const double flops = threads_total * iters * kChains * (kind == 2 ? 4.0 : 2.0);
    for (int rep = 0; rep < 7 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, s);
      if (e != cudaSuccess) break;
      // reps 1-3 one operand pattern, 4-6 the other (rep 0 warms up)
      const bool spread = rep >= 4;
      if (kind == 0)
        spread ? fma_chain_kernel<double, true><<<grid, threads, 0, s>>>(iters, 0.9999999, 1e-7, sink, clk)
               : fma_chain_kernel<double, false><<<grid, threads, 0, s>>>(iters, 0.9999999, 1e-7, sink, clk);
      else if (kind == 1)
        spread ? fma_chain_kernel<float, true><<<grid, threads, 0, s>>>(iters, 0.9999999f, 1e-7f, (float*)sink, clk)
               : fma_chain_kernel<float, false><<<grid, threads, 0, s>>>(iters, 0.9999999f, 1e-7f, (float*)sink, clk);
      else
        fma_chain_f32x2_kernel<<<grid, threads, 0, s>>>(iters, pack2(0.9999999f), pack2(1e-7f), (float*)sink, clk);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      if (rep > 0) best[kind] = std::max(best[kind], flops / (ms * 1e-3) / 1e12);  // rep 0 warms up
      if (kind == 1 && rep == 6) {
        if ((e = cudaMemcpy(hclk.data(), clk, hclk.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost)) !=
            cudaSuccess)
          break;
        std::vector<double> f;
        for (int b = 0; b < grid; ++b)
          if (hclk[2 * b + 1] > 0) f.push_back(1e3 * (double)hclk[2 * b] / (double)hclk[2 * b + 1]);
        if (!f.empty()) {
          std::nth_element(f.begin(), f.begin() + f.size() / 2, f.end());
          mhz = f[f.size() / 2];
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out[0] = best[0];
  out[1] = best[1];
  out[2] = best[2];
  out[3] = mhz;
  return e;
}

}  // namespace kpm
