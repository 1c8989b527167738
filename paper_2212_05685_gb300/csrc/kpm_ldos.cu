// Local density of states of App. C (Eqs. N_i, Gij) from the diagonal
// Chebyshev moments mu_m(I) = [T_m(h~)]_II recorded by the recursion:
//
//   G_II(z) = (1/a) (1/s) sum_{m<M} (2 - delta_m0) w^m mu_m(I),
//   z~ = (z - b)/a, s = sqrt(z~^2 - 1), w = z~ - s with |w| < 1,
//
// the Chebyshev series of the resolvent 1/(z - E) (exact as |w|^M -> 0; no
// damping kernel: the Lorentzian broadening is the imaginary part of z).
// N_i,up(omega) = -(g^t_i,up)^2 Im G_(i,up)(omega + i Gamma)/pi and
// N_i,dn(omega) = -(g^t_i,dn)^2 Im G_(i,dn)(-omega + i Gamma)/pi, Gamma =
// alpha |omega| + Gamma_0.  The sum over m is a dense contraction of the
// n_omega x M coefficient matrix with the M x N moment matrix of each spin:
// one FP64 GEMM per spin (cuBLAS, the library GEMM).
#include <cublas_v2.h>

#include <algorithm>

#include "kpm_internal.cuh"

namespace kpm {
namespace {

constexpr double kPi = 3.14159265358979323846;

// C[sigma][k][m] = Im((2 - delta_m0) w^m / s) / a at z~ of frequency k and spin sigma
__global__ void ldos_coeff_kernel(int M, int nw, const double* __restrict__ omega, double alpha, double gamma0,
                                  const double* __restrict__ ab, double* __restrict__ C) {
  const int64_t total = 2 * (int64_t)nw * M;
  const double a = ab[0], b = ab[1];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(t % M);
    const int64_t r = t / M;
    const int k = (int)(r % nw), sg = (int)(r / nw);
    const double om = sg == 0 ? omega[k] : -omega[k];
    const double gam = alpha * fabs(omega[k]) + gamma0;
    const double zr = (om - b) / a, zi = gam / a;
    // s = sqrt(z^2 - 1), principal branch; then the root with |z - s| < 1
    const double ur = zr * zr - zi * zi - 1.0, ui = 2.0 * zr * zi;
    const double rr = sqrt(hypot(ur, ui));
    const double ph = 0.5 * atan2(ui, ur);
    double sr = rr * cos(ph), si = rr * sin(ph);
    double wr = zr - sr, wi = zi - si;
    if (wr * wr + wi * wi > 1.0) {
      sr = -sr;
      si = -si;
      wr = zr - sr;
      wi = zi - si;
    }
    // w^m = |w|^m e^{i m arg w}
    const double lw = 0.5 * log(wr * wr + wi * wi), aw = atan2(wi, wr);
    const double mag = exp(m * lw);
    double pr, pi;
    sincos(m * aw, &pi, &pr);
    pr *= mag;
    pi *= mag;
    // (pr + i pi) / (sr + i si)
    const double den = sr * sr + si * si;
    const double im = (pi * sr - pr * si) / den;
    C[t] = (m == 0 ? 1.0 : 2.0) * im / a;
  }
}

// ldos[sigma][k][i] *= -weight[sigma][i] / pi (weights null: 1)
__global__ void ldos_scale_kernel(int64_t N, int nw, const double* __restrict__ wgt, double* __restrict__ ldos) {
  const int64_t total = 2 * (int64_t)nw * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % N;
    const int sg = (int)(t / ((int64_t)nw * N));
    ldos[t] *= -(wgt ? wgt[sg * N + i] : 1.0) / kPi;
  }
}

}  // namespace

cudaError_t launch_ldos_coefficients(int M, int nw, const double* omega, double alpha, double gamma0,
                                     const double* ab, double* C, cudaStream_t s) {
  const int64_t total = 2 * (int64_t)nw * M;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 8 * 152));
  ldos_coeff_kernel<<<grid, 256, 0, s>>>(M, nw, omega, alpha, gamma0, ab, C);
  return cudaGetLastError();
}

const char* ldos_contract(void* cublas, int M, int nw, int64_t N, const double* C, const double* rec, double* ldos,
                          const double* wgt, cudaStream_t s) {
  cublasHandle_t h = static_cast<cublasHandle_t>(cublas);
  if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) return "cublasSetStream failed";
  const double one = 1.0, zero = 0.0;
  for (int sg = 0; sg < 2; ++sg) {
    // column-major: out (N x nw, ld N) = mu_sigma (N x M, ld 2N) * C_sigma^T (M x nw, ld M)
    const double* A = rec + sg * N;
    const double* B = C + (int64_t)sg * nw * M;
    double* out = ldos + (int64_t)sg * nw * N;
    if (cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, nw, M, &one, A, (int)(2 * N), B, M, &zero, out, (int)N) !=
        CUBLAS_STATUS_SUCCESS)
      return "cublasDgemm failed";
  }
  const int64_t total = 2 * (int64_t)nw * N;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 8 * 152));
  ldos_scale_kernel<<<grid, 256, 0, s>>>(N, nw, wgt, ldos);
  return cudaGetLastError() == cudaSuccess ? nullptr : "ldos scale kernel failed";
}

void* cublas_create() {
  cublasHandle_t h = nullptr;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return nullptr;
  return h;
}
void cublas_destroy(void* h) {
  if (h) cublasDestroy(static_cast<cublasHandle_t>(h));
}

}  // namespace kpm
