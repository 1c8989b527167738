// FP64 kernels of the self-consistency loop around the KPM pass:
// Peierls phases (Sec. II, App. C), the effective fields of the Gutzwiller
// functional (App. A), Gershgorin rescaling and Chebyshev/Jackson
// coefficients (App. B), observable assembly and the mixing update.
// All O(N); the Chebyshev recursion that dominates the cost is in
// cheb_kernels.cu.
#include <math.h>

#include "kpm_internal.cuh"

namespace kpm {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kClamp = 1e-12;

// forward bonds d and ordered nn pairs e
__constant__ int kFwdX[4] = {1, 0, 1, 1};
__constant__ int kFwdY[4] = {0, 1, 1, -1};
__constant__ int kNnX[4] = {1, 0, -1, 0};
__constant__ int kNnY[4] = {0, 1, 0, -1};

struct Cplx {
  double re, im;
};
__device__ __forceinline__ Cplx cx(double r, double i) { return Cplx{r, i}; }
__device__ __forceinline__ Cplx cadd(Cplx a, Cplx b) { return cx(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ Cplx cmul(Cplx a, Cplx b) {
  return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ Cplx cconj(Cplx a) { return cx(a.re, -a.im); }
__device__ __forceinline__ Cplx cscale(Cplx a, double s) { return cx(a.re * s, a.im * s); }
__device__ __forceinline__ double cabs2(Cplx a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ double cabs(Cplx a) { return hypot(a.re, a.im); }

__device__ __forceinline__ int site_of(int x, int y, int nx, int ny) {
  x %= nx;
  if (x < 0) x += nx;
  y %= ny;
  if (y < 0) y += ny;
  return x + nx * y;
}
__device__ __forceinline__ int shift(int i, int dx, int dy, int nx, int ny) {
  return site_of(i % nx + dx, i / nx + dy, nx, ny);
}

// views of the 26N layout
struct Layout {
  int N;
  __device__ double n(const double* p, int s, int i) const { return p[s * N + i]; }
  __device__ Cplx chi(const double* p, int s, int d, int i) const {
    const double* q = p + 2 * N + 2 * ((s * 4 + d) * N + i);
    return cx(q[0], q[1]);
  }
  __device__ Cplx F(const double* p, int e, int i) const {
    const double* q = p + 18 * N + 2 * (e * N + i);
    return cx(q[0], q[1]);
  }
  __device__ double* n_ptr(double* p, int s, int i) const { return p + s * N + i; }
  __device__ double* chi_ptr(double* p, int s, int d, int i) const {
    return p + 2 * N + 2 * ((s * 4 + d) * N + i);
  }
  __device__ double* F_ptr(double* p, int e, int i) const { return p + 18 * N + 2 * (e * N + i); }
};

// Gutzwiller site factors (App. A) and their derivatives with respect to
// n_{i up}, n_{i dn} (delta = 1 - n_up - n_dn, m = (n_up - n_dn)/2).
struct SiteF {
  double delta, m, P;
  double gt[2], dgt[2][2];  // dgt[s][s'] = d g^t_s / d n_s'
  double gxy, dgxy[2];
};

__device__ SiteF site_factors(double nu, double nd, bool gutz) {
  SiteF f;
  f.delta = 1.0 - nu - nd;
  f.m = 0.5 * (nu - nd);
  f.P = 1.0 - f.delta * f.delta + 4.0 * f.m * f.m;
  if (!gutz) {
    f.gt[0] = f.gt[1] = 1.0;
    f.dgt[0][0] = f.dgt[0][1] = f.dgt[1][0] = f.dgt[1][1] = 0.0;
    f.gxy = 1.0;
    f.dgxy[0] = f.dgxy[1] = 0.0;
    return f;
  }
  const bool clamped = f.delta <= kClamp;
  const double de = clamped ? kClamp : f.delta;
  const double m = f.m;
  const double Pe = 1.0 - de * de + 4.0 * m * m;
  for (int s = 0; s < 2; ++s) {
    const double sg = s == 0 ? 1.0 : -1.0;
    const double up = 1.0 + de + 2.0 * sg * m;
    const double dn = 1.0 + de - 2.0 * sg * m;
    const double g = sqrt(2.0 * de * (1.0 - de) / Pe * up / dn);
    double dld = 1.0 / de - 1.0 / (1.0 - de) + 2.0 * de / Pe + 1.0 / up - 1.0 / dn;
    if (clamped) dld = 0.0;
    const double dlm = -8.0 * m / Pe + 2.0 * sg / up + 2.0 * sg / dn;
    f.gt[s] = g;
    f.dgt[s][0] = 0.5 * g * (-dld + 0.5 * dlm);
    f.dgt[s][1] = 0.5 * g * (-dld - 0.5 * dlm);
  }
  f.gxy = 2.0 * (1.0 - f.delta) / f.P;
  const double ld = -1.0 / (1.0 - f.delta) + 2.0 * f.delta / f.P;
  const double lm = -8.0 * m / f.P;
  f.dgxy[0] = f.gxy * (-ld + 0.5 * lm);
  f.dgxy[1] = f.gxy * (-ld - 0.5 * lm);
  return f;
}

// Exchange term of one nn bond (i, j): W_b = J [g^z (m_i m_j - S/4) - g^xy Q]
// with g^z = g^xy R, R = (A - c X^2)/(A - c), A = 2(|Dbar|^2 - |chibar|^2),
// c = 4 m_i m_j (App. A; reading W3), and the derivative pieces.
struct BondX {
  double gxy, gz, R, dRA, dRc, dRX, Ez, Q, W;
  double dX_ddi, dX_ddj, dX_dmi, dX_dmj;
  Cplx chib, delb;
};

__device__ BondX bond_exchange(const SiteF& a, const SiteF& b, Cplx cu, Cplx cd, Cplx Fij, Cplx Fji,
                               double J, bool gutz) {
  BondX o;
  o.gxy = a.gxy * b.gxy;
  const double S = cabs2(cu) + cabs2(cd) + cabs2(Fij) + cabs2(Fji);
  o.Q = cmul(cu, cconj(cd)).re + cmul(cconj(Fij), Fji).re;
  o.Ez = J * (a.m * b.m - 0.25 * S);
  if (gutz) {
    o.chib = cscale(cadd(cu, cd), 0.5);
    o.delb = cscale(cadd(Fij, Fji), 0.5);
    const double A = 2.0 * (cabs2(o.delb) - cabs2(o.chib));
    const double c = 4.0 * a.m * b.m;
    const double X = 1.0 + 12.0 * (1.0 - a.delta) * (1.0 - b.delta) / sqrt(a.P * b.P);
    if (c == 0.0) {
      o.R = 1.0;
      o.dRA = 0.0;
      o.dRX = 0.0;
      o.dRc = A == 0.0 ? 0.0 : (1.0 - X * X) / A;
    } else {
      const double den = A - c;
      o.R = (A - c * X * X) / den;
      o.dRA = c * (X * X - 1.0) / (den * den);
      o.dRc = A * (1.0 - X * X) / (den * den);
      o.dRX = -2.0 * c * X / den;
    }
    const double Xm1 = X - 1.0;
    o.dX_ddi = Xm1 * (-1.0 / (1.0 - a.delta) + a.delta / a.P);
    o.dX_ddj = Xm1 * (-1.0 / (1.0 - b.delta) + b.delta / b.P);
    o.dX_dmi = Xm1 * (-4.0 * a.m / a.P);
    o.dX_dmj = Xm1 * (-4.0 * b.m / b.P);
  } else {
    o.chib = o.delb = cx(0.0, 0.0);
    o.R = 1.0;
    o.dRA = o.dRc = o.dRX = 0.0;
    o.dX_ddi = o.dX_ddj = o.dX_dmi = o.dX_dmj = 0.0;
  }
  o.gz = o.gxy * o.R;
  o.W = J * (o.gz * (a.m * b.m - 0.25 * S) - o.gxy * o.Q);
  return o;
}

// d W_b / d n_{sp} of one end of the bond; `self` is that end, `other` the
// opposite end, first=true when `self` is the bond's first site.
__device__ double bond_dn(const BondX& b, const SiteF& self, const SiteF& other, int sp, bool first,
                          double J) {
  const double h = sp == 0 ? 0.5 : -0.5;  // dm/dn_sp
  const double dWdgxy = b.Ez * b.R - J * b.Q;
  const double dWdR = b.Ez * b.gxy;
  const double dX_dd = first ? b.dX_ddi : b.dX_ddj;
  const double dX_dm = first ? b.dX_dmi : b.dX_dmj;
  return J * b.gz * other.m * h + dWdgxy * other.gxy * self.dgxy[sp] +
         dWdR * (b.dRc * 4.0 * other.m * h + b.dRX * (-dX_dd + h * dX_dm));
}

__global__ void peierls_kernel(kpm_model m, double* phi) {
  const int N = m.nx * m.ny;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int x = i % m.nx, y = i / m.nx;
  const double f = 2.0 * kPi * m.flux / ((double)m.nx * m.ny);
  for (int d = 0; d < 4; ++d) {
    const int dx = kFwdX[d], dy = kFwdY[d];
    // -(pi/Phi0) B * integral x dy along the straight bond
    double p = -f * dy * (x + 0.5 * dx);
    if (x + dx >= m.nx) {  // bond crosses the x boundary: magnetic translation phase
      int yy = (y + dy) % m.ny;
      if (yy < 0) yy += m.ny;
      p += 2.0 * kPi * m.flux * yy / m.ny;
    }
    phi[d * N + i] = p;
  }
}

// One thread per site: T and D on the bonds stored at site i, eps_i from the
// eight bonds that touch i, and the site's share of W (its forward bonds).
__global__ void fields_kernel(kpm_model m, const double* __restrict__ phi,
                              const double* __restrict__ p, double mu, double* __restrict__ fld,
                              double* __restrict__ wsite) {
  const int nx = m.nx, ny = m.ny, N = nx * ny;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const Layout L{N};
  const bool gutz = m.gutzwiller != 0;
  const double J = m.J;
  const double tamp[4] = {m.t, m.t, m.tp, m.tp};

  const SiteF si = site_factors(L.n(p, 0, i), L.n(p, 1, i), gutz);
  double eps[2] = {-mu, -mu};
  Cplx T[2][4];
  Cplx Dv[4];
  for (int s = 0; s < 2; ++s)
    for (int d = 0; d < 4; ++d) T[s][d] = cx(0.0, 0.0);
  for (int e = 0; e < 4; ++e) Dv[e] = cx(0.0, 0.0);
  double W = 0.0;

  // hopping on forward bonds i -> j
  for (int d = 0; d < 4; ++d) {
    const int j = shift(i, kFwdX[d], kFwdY[d], nx, ny);
    const SiteF sj = site_factors(L.n(p, 0, j), L.n(p, 1, j), gutz);
    double sn, cs;
    sincos(phi[d * N + i], &sn, &cs);
    const Cplx tij = cx(tamp[d] * cs, tamp[d] * sn);
    for (int s = 0; s < 2; ++s) {
      const double gg = si.gt[s] * sj.gt[s];
      T[s][d] = cadd(T[s][d], cscale(tij, -gg));
      const double e2 = 2.0 * cmul(tij, L.chi(p, s, d, i)).re;
      W -= gg * e2;
      for (int sp = 0; sp < 2; ++sp) eps[sp] -= si.dgt[s][sp] * sj.gt[s] * e2;
    }
  }
  // hopping on bonds k -> i that end at i
  for (int d = 0; d < 4; ++d) {
    const int k = shift(i, -kFwdX[d], -kFwdY[d], nx, ny);
    const SiteF sk = site_factors(L.n(p, 0, k), L.n(p, 1, k), gutz);
    double sn, cs;
    sincos(phi[d * N + k], &sn, &cs);
    const Cplx tki = cx(tamp[d] * cs, tamp[d] * sn);
    for (int s = 0; s < 2; ++s) {
      const double e2 = 2.0 * cmul(tki, L.chi(p, s, d, k)).re;
      for (int sp = 0; sp < 2; ++sp) eps[sp] -= si.dgt[s][sp] * sk.gt[s] * e2;
    }
  }
  // exchange on nn bonds starting at i: (i, j = i + d)
  for (int d = 0; d < 2; ++d) {
    const int j = shift(i, kFwdX[d], kFwdY[d], nx, ny);
    const SiteF sj = site_factors(L.n(p, 0, j), L.n(p, 1, j), gutz);
    const Cplx cu = L.chi(p, 0, d, i), cd = L.chi(p, 1, d, i);
    const Cplx Fij = L.F(p, d, i), Fji = L.F(p, d + 2, j);
    const BondX b = bond_exchange(si, sj, cu, cd, Fij, Fji, J, gutz);
    W += b.W;
    const double coefA = b.Ez * b.gxy * b.dRA;
    const Cplx cbc = cconj(b.chib);
    T[0][d] = cadd(T[0][d], cadd(cscale(cadd(cscale(cconj(cu), -0.25 * b.gz), cscale(cconj(cd), -0.5 * b.gxy)), J),
                                 cscale(cbc, -coefA)));
    T[1][d] = cadd(T[1][d], cadd(cscale(cadd(cscale(cconj(cd), -0.25 * b.gz), cscale(cconj(cu), -0.5 * b.gxy)), J),
                                 cscale(cbc, -coefA)));
    Dv[d] = cadd(Dv[d], cadd(cscale(cadd(cscale(Fij, -0.25 * b.gz), cscale(Fji, -0.5 * b.gxy)), J),
                             cscale(b.delb, coefA)));
    for (int sp = 0; sp < 2; ++sp) eps[sp] += bond_dn(b, si, sj, sp, true, J);
  }
  // exchange on nn bonds ending at i: (k = i - d, i); D_{i,k} is stored at e = d + 2
  for (int d = 0; d < 2; ++d) {
    const int k = shift(i, -kFwdX[d], -kFwdY[d], nx, ny);
    const SiteF sk = site_factors(L.n(p, 0, k), L.n(p, 1, k), gutz);
    const Cplx cu = L.chi(p, 0, d, k), cd = L.chi(p, 1, d, k);
    const Cplx Fki = L.F(p, d, k), Fik = L.F(p, d + 2, i);
    const BondX b = bond_exchange(sk, si, cu, cd, Fki, Fik, J, gutz);
    const double coefA = b.Ez * b.gxy * b.dRA;
    Dv[d + 2] = cadd(Dv[d + 2], cadd(cscale(cadd(cscale(Fik, -0.25 * b.gz), cscale(Fki, -0.5 * b.gxy)), J),
                                     cscale(b.delb, coefA)));
    for (int sp = 0; sp < 2; ++sp) eps[sp] += bond_dn(b, si, sk, sp, false, J);
  }

  *L.n_ptr(fld, 0, i) = eps[0];
  *L.n_ptr(fld, 1, i) = eps[1];
  for (int s = 0; s < 2; ++s)
    for (int d = 0; d < 4; ++d) {
      double* q = L.chi_ptr(fld, s, d, i);
      q[0] = T[s][d].re;
      q[1] = T[s][d].im;
    }
  for (int e = 0; e < 4; ++e) {
    double* q = L.F_ptr(fld, e, i);
    q[0] = Dv[e].re;
    q[1] = Dv[e].im;
  }
  if (wsite) wsite[i] = W - mu * (L.n(p, 0, i) + L.n(p, 1, i));
}

// ---------------------------------------------------------------- reductions
// Two-stage, fixed-order reductions (deterministic results run to run).
constexpr int kRedGrid = 512;

template <int OP>  // 0 sum, 1 max, 2 min
__device__ double red_op(double a, double b) {
  return OP == 0 ? a + b : (OP == 1 ? fmax(a, b) : fmin(a, b));
}
template <int OP>
__device__ double red_init() {
  return OP == 0 ? 0.0 : (OP == 1 ? -INFINITY : INFINITY);
}

template <int OP>
__device__ double block_reduce(double v) {
  __shared__ double sm[kRedBlock / 32];
  for (int o = 16; o > 0; o >>= 1) v = red_op<OP>(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sm[lane] : red_init<OP>();
    for (int o = 16; o > 0; o >>= 1) v = red_op<OP>(v, __shfl_down_sync(0xffffffffu, v, o));
  }
  __syncthreads();
  return v;
}

template <int OP>
__global__ void reduce_partial(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  double v = red_init<OP>();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    v = red_op<OP>(v, x[k]);
  v = block_reduce<OP>(v);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

template <int OP>
__global__ void reduce_final(const double* __restrict__ part, int n, double* __restrict__ out,
                             const double* __restrict__ scale) {
  double v = red_init<OP>();
  for (int k = threadIdx.x; k < n; k += blockDim.x) v = red_op<OP>(v, part[k]);
  v = block_reduce<OP>(v);
  if (threadIdx.x == 0) *out = scale ? v * *scale : v;
}

int grid_for(int64_t n) {
  int64_t g = (n + kRedBlock - 1) / kRedBlock;
  if (g < 1) g = 1;
  if (g > kRedGrid) g = kRedGrid;
  return (int)g;
}

// eps -= mean(eps) + mu_eff ; mu_out = mu_eff + mean
__global__ void shift_eps_kernel(int N, double* __restrict__ fld, const double* __restrict__ mean_sum,
                                 const double* __restrict__ mu_eff, double* __restrict__ mu_out) {
  const double mean = *mean_sum / (2.0 * N);
  const double sh = mean + *mu_eff;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 2 * N; k += gridDim.x * blockDim.x) fld[k] -= sh;
  if (blockIdx.x == 0 && threadIdx.x == 0 && mu_out) *mu_out = *mu_eff + mean;
}

// Gershgorin row bounds: per site the max of h_II + R_I and min of h_II - R_I
__global__ void gershgorin_partial(kpm_model m, const double* __restrict__ fld, double* __restrict__ part) {
  const int nx = m.nx, ny = m.ny, N = nx * ny;
  const Layout L{N};
  double hi = -INFINITY, lo = INFINITY;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double R0 = 0.0, R1 = 0.0;
    for (int d = 0; d < 4; ++d) {
      const int k = shift(i, -kFwdX[d], -kFwdY[d], nx, ny);
      R0 += cabs(L.chi(fld, 0, d, i)) + cabs(L.chi(fld, 0, d, k));
      R1 += cabs(L.chi(fld, 1, d, i)) + cabs(L.chi(fld, 1, d, k));
    }
    for (int e = 0; e < 4; ++e) {
      const int j = shift(i, kNnX[e], kNnY[e], nx, ny);
      R0 += cabs(L.F(fld, e, i));
      R1 += cabs(L.F(fld, (e + 2) & 3, j));
    }
    const double d0 = L.n(fld, 0, i), d1 = -L.n(fld, 1, i);
    hi = fmax(hi, fmax(d0 + R0, d1 + R1));
    lo = fmin(lo, fmin(d0 - R0, d1 - R1));
  }
  hi = block_reduce<1>(hi);
  lo = block_reduce<2>(lo);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = hi;
    part[2 * blockIdx.x + 1] = lo;
  }
}

__global__ void gershgorin_final(const double* __restrict__ part, int n, double margin, int symmetric,
                                 double* __restrict__ ab) {
  double hi = -INFINITY, lo = INFINITY;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    hi = fmax(hi, part[2 * k]);
    lo = fmin(lo, part[2 * k + 1]);
  }
  hi = block_reduce<1>(hi);
  lo = block_reduce<2>(lo);
  if (threadIdx.x == 0) {
    if (symmetric) {  // particle-hole symmetric spectrum: centre 0, half-width max(hi, -lo)
      const double half = fmax(hi, -lo);
      ab[0] = half > 0.0 ? (1.0 + margin) * half : 1.0;
      ab[1] = 0.0;
    } else {
      const double half = 0.5 * (hi - lo);
      ab[0] = half > 0.0 ? (1.0 + margin) * half : 1.0;
      ab[1] = 0.5 * (hi + lo);
    }
  }
}

// Largest deviation of the fields from the particle-hole symmetric sector
// (eps_up = eps_dn, T_up = T_dn, D_ij = D_ji) and the largest field modulus:
// part[2 b] = deviation, part[2 b + 1] = modulus for block b.
__global__ void ph_asym_partial(kpm_model m, const double* __restrict__ fld, double* __restrict__ part) {
  const int nx = m.nx, ny = m.ny, N = nx * ny;
  const Layout L{N};
  double dev = 0.0, mag = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double e0 = L.n(fld, 0, i), e1 = L.n(fld, 1, i);
    dev = fmax(dev, fabs(e0 - e1));
    mag = fmax(mag, fmax(fabs(e0), fabs(e1)));
    for (int d = 0; d < 4; ++d) {
      const Cplx t0 = L.chi(fld, 0, d, i), t1 = L.chi(fld, 1, d, i);
      dev = fmax(dev, cabs(cx(t0.re - t1.re, t0.im - t1.im)));
      mag = fmax(mag, fmax(cabs(t0), cabs(t1)));
    }
    for (int e = 0; e < 4; ++e) {
      const int j = shift(i, kNnX[e], kNnY[e], nx, ny);
      const Cplx a = L.F(fld, e, i), b = L.F(fld, (e + 2) & 3, j);
      dev = fmax(dev, cabs(cx(a.re - b.re, a.im - b.im)));
      mag = fmax(mag, cabs(a));
    }
  }
  dev = block_reduce<1>(dev);
  mag = block_reduce<1>(mag);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = dev;
    part[2 * blockIdx.x + 1] = mag;
  }
}

// Jackson-damped Chebyshev coefficients of the T = 0 step theta(x0 - x) and
// of min(x - x0, 0), x0 = -b/a (App. B, Eqs. rho_KPM and F_KPM; reading K2).
__device__ double S_theta(int k, double th) {  // int_{th}^{pi} cos(k t) dt
  k = k < 0 ? -k : k;
  return k == 0 ? kPi - th : -sin(k * th) / k;
}

// half: particle-hole half pass, where the grand potential's diagonal moments of
// the columns (j, dn) equal (-1)^m those of (j, up): a^Omega_m (1 + (-1)^m)
__global__ void coefficients_kernel(int M, const double* __restrict__ ab, double* __restrict__ am,
                                    double* __restrict__ ao, int half) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double x0 = -ab[1] / ab[0];
  x0 = fmin(1.0, fmax(-1.0, x0));
  const double th = acos(x0);
  const double q = kPi / (M + 1);
  const double g = ((M - m + 1) * cos(q * m) + sin(q * m) * cos(q) / sin(q)) / (M + 1);
  const double c = m == 0 ? 1.0 - th / kPi : -sin(m * th) / (m * kPi);
  const double co = (0.5 * (S_theta(m + 1, th) + S_theta(m - 1, th)) - x0 * S_theta(m, th)) / kPi;
  const double w = m == 0 ? 1.0 : 2.0;
  am[m] = w * g * c;
  ao[m] = half ? ((m & 1) ? 0.0 : 2.0 * w * g * co) : w * g * co;
}

// Per-site table of 2h~ = 2(h - b)/a (App. B rescaling), neighbour order
//   k = 1..8 : (+1,0) (-1,0) (0,+1) (0,-1) (+1,+1) (-1,-1) (+1,-1) (-1,+1)
// [0]      : (2(eps_up - b)/a, 2(-eps_dn - b)/a)        (diagonals, packed)
// [1..8]   : row (i,0) -> (j_k, 0)
// [9..16]  : row (i,1) -> (j_k, 1)
// [17..20] : row (i,0) -> (j_k, 1), k = 1..4
// [21..24] : row (i,1) -> (j_k, 0), k = 1..4
// [25]     : 0 (padding to 16-byte multiples)
template <typename C>
__device__ __forceinline__ C to_c(Cplx v);
template <>
__device__ __forceinline__ float2 to_c<float2>(Cplx v) { return make_float2((float)v.re, (float)v.im); }
template <>
__device__ __forceinline__ double2 to_c<double2>(Cplx v) { return make_double2(v.re, v.im); }
// double-float: each FP64 part as hi + lo with lo the rounding residual of hi
template <>
__device__ __forceinline__ float4 to_c<float4>(Cplx v) {
  const float rh = __double2float_rn(v.re), ih = __double2float_rn(v.im);
  return make_float4(rh, __double2float_rn(v.re - (double)rh), ih, __double2float_rn(v.im - (double)ih));
}


template <typename C>
__global__ void scale_table_kernel(kpm_model m, const double* __restrict__ fld, const double* __restrict__ ab,
                                   C* __restrict__ table) {
  const int nx = m.nx, ny = m.ny, N = nx * ny;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const Layout L{N};
  const double a = ab[0], b = ab[1];
  const double s = 2.0 / a;
  C* out = table + (size_t)i * kCoef;
  out[0] = to_c<C>(cx(2.0 * (L.n(fld, 0, i) - b) / a, 2.0 * (-L.n(fld, 1, i) - b) / a));
  // forward bond d for neighbours k = 1,3,5,7 and backward for k = 2,4,6,8
  const int dir_of_k[8] = {0, 0, 1, 1, 2, 2, 3, 3};
  for (int k = 0; k < 8; ++k) {
    const int d = dir_of_k[k];
    Cplx up, dn;
    if ((k & 1) == 0) {  // forward: i -> i + d
      up = L.chi(fld, 0, d, i);
      dn = cscale(cconj(L.chi(fld, 1, d, i)), -1.0);
    } else {             // backward: i -> i - d, conjugate of the bond stored at i - d
      const int j = shift(i, -kFwdX[d], -kFwdY[d], nx, ny);
      up = cconj(L.chi(fld, 0, d, j));
      dn = cscale(L.chi(fld, 1, d, j), -1.0);
    }
    out[1 + k] = to_c<C>(cscale(up, s));
    out[9 + k] = to_c<C>(cscale(dn, s));
  }
  // nn neighbours k = 1..4 in the order (+1,0) (-1,0) (0,+1) (0,-1) -> e = 0, 2, 1, 3
  const int e_of_k[4] = {0, 2, 1, 3};
  for (int k = 0; k < 4; ++k) {
    const int e = e_of_k[k];
    const int j = shift(i, kNnX[e], kNnY[e], nx, ny);
    out[17 + k] = to_c<C>(cscale(L.F(fld, e, i), -s));
    out[21 + k] = to_c<C>(cscale(cconj(L.F(fld, (e + 2) & 3, j)), -s));
  }
  out[25] = to_c<C>(cx(0.0, 0.0));
}

// Observables from the accumulated entries of F_M(h~) e_J (readings N2, N3):
//   column (j,0): n_up = acc[0], chi_up[d] = acc[1+d], F[e] = -conj(acc[5+e])
//   column (j,1): n_dn = 1 - acc[0], chi_dn[d] = -conj(acc[1+d])
// half: only the columns (j,0) were propagated; in the particle-hole symmetric
// sector F_M(h~) = 1 - U conj(F_M(h~)) U^T (U: (c_up, c^dag_dn) -> (c_dn,
// -c^dag_up) per site), so column (j,1) gives n_dn = n_up, chi_dn = chi_up, and
// acc[(j,0)][9] already holds both diagonal Omega moments.
// Sites outside [sb, se) (a pass over part of the columns) get zero order
// parameters and add nothing to Omega.
__global__ void assemble_kernel(int nx, int ny, const double2* __restrict__ acc, double* __restrict__ obs,
                                double* __restrict__ part, int half, int sb, int se) {
  const int N = nx * ny;
  const Layout L{N};
  double om = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    if (j < sb || j >= se) {
      for (int s = 0; s < 2; ++s) *L.n_ptr(obs, s, j) = 0.0;
      for (int s = 0; s < 2; ++s)
        for (int d = 0; d < 4; ++d) {
          double* q = L.chi_ptr(obs, s, d, j);
          q[0] = q[1] = 0.0;
        }
      for (int e = 0; e < 4; ++e) {
        double* q = L.F_ptr(obs, e, j);
        q[0] = q[1] = 0.0;
      }
      continue;
    }
    const double2* a0 = acc + (size_t)(2 * j) * kSlots;
    const double2* a1 = acc + (size_t)(2 * j + 1) * kSlots;
    *L.n_ptr(obs, 0, j) = a0[0].x;
    *L.n_ptr(obs, 1, j) = half ? a0[0].x : 1.0 - a1[0].x;
    for (int d = 0; d < 4; ++d) {
      double* q0 = L.chi_ptr(obs, 0, d, j);
      q0[0] = a0[1 + d].x;
      q0[1] = a0[1 + d].y;
      double* q1 = L.chi_ptr(obs, 1, d, j);
      q1[0] = half ? a0[1 + d].x : -a1[1 + d].x;
      q1[1] = half ? a0[1 + d].y : a1[1 + d].y;
    }
    for (int e = 0; e < 4; ++e) {
      double* q = L.F_ptr(obs, e, j);
      if (half) {
        // singlet sector: F_{j,j+e} = F_{j+e,j}; the two estimates (columns
        // (j, up) and (j+e, up)) are averaged, which keeps the state exactly in
        // the sector the half pass assumes
        const int k = shift(j, kNnX[e], kNnY[e], nx, ny);
        const double2 b = acc[(size_t)(2 * k) * kSlots + 5 + ((e + 2) & 3)];
        q[0] = 0.5 * (-a0[5 + e].x - b.x);
        q[1] = 0.5 * (a0[5 + e].y + b.y);
      } else {
        q[0] = -a0[5 + e].x;
        q[1] = a0[5 + e].y;
      }
    }
    om += half ? a0[9].x : a0[9].x + a1[9].x;
  }
  om = block_reduce<0>(om);
  if (threadIdx.x == 0) part[blockIdx.x] = om;
}

// Mixing update (readings R1, R2): part 1 per site for the densities
// (paramagnetic average, projection onto <n> = n_target), part 2 for the
// complex parameters.  Writes the per-block max |p_new - p| into part.
// rec (optional): per-call record of the loop, {a, b, mu, omega, residual,
// density error, iterations, frozen, ...}; once an iteration met tol (or
// turned non-finite) `frozen` is set and later iterations leave every output
// as it is, so queuing iterations past convergence changes nothing.
__device__ __forceinline__ bool frozen(const double* rec) { return rec != nullptr && rec[7] != 0.0; }

__global__ void update_kernel(int N, double* __restrict__ p, double* __restrict__ o,
                              const double* __restrict__ nsum, kpm_rmft_opts opt, double* __restrict__ part,
                              const double* __restrict__ rec) {
  if (frozen(rec)) return;
  const double e = *nsum / N - opt.n_target;
  double r = 0.0;
  const int64_t total = (int64_t)N + 24 * (int64_t)N;  // N site pairs, then 24N complex reals
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    if (k < N) {
      const int i = (int)k;
      double ou = o[i], od = o[N + i];
      if (opt.paramagnetic) ou = od = 0.5 * (ou + od);
      ou -= 0.5 * e;
      od -= 0.5 * e;
      const double pu = p[i], pd = p[N + i];
      r = fmax(r, fmax(fabs(ou - pu), fabs(od - pd)));
      p[i] = (1.0 - opt.alpha_n) * pu + opt.alpha_n * ou;
      p[N + i] = (1.0 - opt.alpha_n) * pd + opt.alpha_n * od;
      o[i] = ou;
      o[N + i] = od;
    } else {
      const int64_t q = 2 * (int64_t)N + (k - N);
      const double pv = p[q], ov = o[q];
      r = fmax(r, fabs(ov - pv));
      p[q] = (1.0 - opt.alpha) * pv + opt.alpha * ov;
    }
  }
  // NaN propagates through fmax only if both are NaN; make it sticky
  r = block_reduce<1>(r != r ? INFINITY : r);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// the record of one finished iteration: stats of its pass (snap = {a, b, mu,
// omega}), residual r, density error e, count; freezes on tol or non-finite
__device__ void record_iteration(double* rec, const double* snap, double r, double e, double tol) {
  for (int k = 0; k < 4; ++k) rec[k] = snap[k];
  rec[4] = r;
  rec[5] = e;
  rec[6] += 1.0;
  const bool bad = !(r == r) || r > 1e300 || !(snap[3] == snap[3]);
  if (bad || (r < tol && fabs(e) < tol)) rec[7] = 1.0;
}

__global__ void update_final(const double* __restrict__ part, int n, int N, const double* __restrict__ nsum,
                             kpm_rmft_opts opt, double* __restrict__ mu_eff, double* __restrict__ stats,
                             double* __restrict__ rec, const double* __restrict__ snap) {
  if (frozen(rec)) return;
  double r = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) r = fmax(r, part[k]);
  r = block_reduce<1>(r);
  if (threadIdx.x == 0) {
    const double e = *nsum / N - opt.n_target;
    stats[0] = r;
    stats[1] = e;
    *mu_eff = *mu_eff - opt.eta * e;
    if (rec) record_iteration(rec, snap, r, e, opt.tol);
  }
}

// ---- Anderson (Pulay) mixing, reading R4 -----------------------------------
// State x = (params, mu_eff) of length L = 26 N + 1; preconditioned residual
// f = B (G(x) - x) with B the linear mixings (alpha_n on the densities, alpha
// on chi and F) and f_mu = -eta e; history of the last m differences dX, dF
// (ring, slot (k - 1) mod m at Anderson iteration k); gamma = argmin
// |f - dF gamma|_2 with the normal equations regularised by 1e-10 tr/nh;
// x <- x + f - (dX + dF) gamma.
__global__ void anderson_resid_kernel(int N, const double* __restrict__ p, double* __restrict__ o,
                                      const double* __restrict__ nsum, const double* __restrict__ mu_eff,
                                      kpm_rmft_opts opt, int m, double* __restrict__ xprev, double* __restrict__ fprev,
                                      double* __restrict__ fcur, double* __restrict__ dX, double* __restrict__ dF,
                                      double* __restrict__ part, const double* __restrict__ rec) {
  if (frozen(rec)) return;
  const double e = *nsum / N - opt.n_target;
  const int k = (int)rec[8];
  const int64_t L = 26 * (int64_t)N + 1;
  const int64_t slot = k >= 1 ? (int64_t)((k - 1) % m) * L : -1;
  double r = 0.0;
  auto put = [&](int64_t q, double x, double f) {
    if (slot >= 0) {
      dX[slot + q] = x - xprev[q];
      dF[slot + q] = f - fprev[q];
    }
    xprev[q] = x;
    fprev[q] = f;
    fcur[q] = f;
  };
  const int64_t items = (int64_t)N + 24 * (int64_t)N + 1;  // N site pairs, 24 N complex reals, mu_eff
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < N) {
      const int i = (int)t;
      double ou = o[i], od = o[N + i];
      if (opt.paramagnetic) ou = od = 0.5 * (ou + od);
      ou -= 0.5 * e;
      od -= 0.5 * e;
      const double pu = p[i], pd = p[N + i];
      r = fmax(r, fmax(fabs(ou - pu), fabs(od - pd)));
      o[i] = ou;
      o[N + i] = od;
      put(i, pu, opt.alpha_n * (ou - pu));
      put(N + i, pd, opt.alpha_n * (od - pd));
    } else if (t < items - 1) {
      const int64_t q = 2 * (int64_t)N + (t - N);
      const double pv = p[q], ov = o[q];
      r = fmax(r, fabs(ov - pv));
      put(q, pv, opt.alpha * (ov - pv));
    } else {
      put(L - 1, *mu_eff, -opt.eta * e);
    }
  }
  r = block_reduce<1>(r != r ? INFINITY : r);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

constexpr int kAndChunks = 16;  // column chunks of the Gram sums

// partial dot products: blockIdx.x = pair (a, b) with a <= b < m, or (a, m)
// for <dF_a, f>; blockIdx.y = chunk of the L entries
__global__ void anderson_gram_kernel(int64_t L, int m, const double* __restrict__ dF, const double* __restrict__ fcur,
                                     double* __restrict__ gpart, const double* __restrict__ rec) {
  if (frozen(rec)) return;
  int a = 0, b = 0, t = blockIdx.x;
  for (a = 0; a < m; ++a) {
    const int row = m + 1 - a;  // pairs (a, a..m)
    if (t < row) {
      b = a + t;
      break;
    }
    t -= row;
  }
  const double* u = dF + (int64_t)a * L;
  const double* v = b < m ? dF + (int64_t)b * L : fcur;
  const int64_t chunk = (L + kAndChunks - 1) / kAndChunks;
  const int64_t lo = blockIdx.y * chunk, hi = min(L, lo + chunk);
  double acc = 0.0;
  for (int64_t q = lo + threadIdx.x; q < hi; q += blockDim.x) acc += u[q] * v[q];
  acc = block_reduce<0>(acc);
  if (threadIdx.x == 0) gpart[(int64_t)blockIdx.x * kAndChunks + blockIdx.y] = acc;
}

// gamma from the regularised normal equations (Cholesky, nh <= 16 unknowns);
// gamma = 0 when there is no history or the factorisation fails
__global__ void anderson_solve_kernel(int m, const double* __restrict__ gpart, double* __restrict__ gamma,
                                      const double* __restrict__ rec) {
  if (frozen(rec) || threadIdx.x != 0) return;
  const int nh = min((int)rec[8], m);
  double G[16][16], rhs[16];
  int t = 0;
  for (int a = 0; a < m; ++a)
    for (int b = a; b <= m; ++b, ++t) {
      double v = 0.0;
      for (int c = 0; c < kAndChunks; ++c) v += gpart[(int64_t)t * kAndChunks + c];
      if (a < nh && b < nh) G[a][b] = G[b][a] = v;
      if (a < nh && b == m) rhs[a] = v;
    }
  for (int a = 0; a < m; ++a) gamma[a] = 0.0;
  if (nh == 0) return;
  double tr = 0.0;
  for (int a = 0; a < nh; ++a) tr += G[a][a];
  if (!(tr > 0.0) || !(tr < 1e300)) return;
  const double reg = 1e-10 * tr / nh;
  for (int a = 0; a < nh; ++a) G[a][a] += reg;
  // Cholesky G = C C^T in place (lower triangle)
  for (int j = 0; j < nh; ++j) {
    double d = G[j][j];
    for (int k = 0; k < j; ++k) d -= G[j][k] * G[j][k];
    if (!(d > 0.0)) return;
    const double cjj = sqrt(d);
    G[j][j] = cjj;
    for (int i = j + 1; i < nh; ++i) {
      double v = G[i][j];
      for (int k = 0; k < j; ++k) v -= G[i][k] * G[j][k];
      G[i][j] = v / cjj;
    }
  }
  double y[16];
  for (int i = 0; i < nh; ++i) {
    double v = rhs[i];
    for (int k = 0; k < i; ++k) v -= G[i][k] * y[k];
    y[i] = v / G[i][i];
  }
  for (int i = nh - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < nh; ++k) v -= G[k][i] * gamma[k];
    gamma[i] = v / G[i][i];
  }
}

__global__ void anderson_apply_kernel(int N, double* __restrict__ p, double* __restrict__ mu_eff, int m,
                                      const double* __restrict__ fcur, const double* __restrict__ dX,
                                      const double* __restrict__ dF, const double* __restrict__ gamma,
                                      const double* __restrict__ rec) {
  if (frozen(rec)) return;
  const int64_t L = 26 * (int64_t)N + 1;
  const int nh = min((int)rec[8], m);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L; q += (int64_t)gridDim.x * blockDim.x) {
    double* x = q < L - 1 ? p + q : mu_eff;
    double v = *x + fcur[q];
    for (int a = 0; a < nh; ++a) v -= gamma[a] * (dX[(int64_t)a * L + q] + dF[(int64_t)a * L + q]);
    *x = v;
  }
}

__global__ void anderson_final(const double* __restrict__ part, int n, int N, const double* __restrict__ nsum,
                               kpm_rmft_opts opt, double* __restrict__ stats, double* __restrict__ rec,
                               const double* __restrict__ snap) {
  if (frozen(rec)) return;
  double r = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) r = fmax(r, part[k]);
  r = block_reduce<1>(r);
  if (threadIdx.x == 0) {
    const double e = *nsum / N - opt.n_target;
    stats[0] = r;
    stats[1] = e;
    rec[8] += 1.0;
    record_iteration(rec, snap, r, e, opt.tol);
  }
}

// dL/dphi of the bond i -> i + d through T_{ij s} = -g^t_ij s t_ij e^{i phi} + ...
// and through the site energies at both ends (the g^t derivative terms hold
// 2 Re(t_ij chi_ij s)).  One thread per site and forward bond.
__global__ void phi_grad_kernel(kpm_model m, const double* __restrict__ phi, const double* __restrict__ p,
                                const double* __restrict__ gf, double* __restrict__ out) {
  const int nx = m.nx, ny = m.ny, N = nx * ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * N) return;
  const int d = t / N, i = t - d * N;
  const Layout L{N};
  const bool gutz = m.gutzwiller != 0;
  const double tamp = d < 2 ? m.t : m.tp;
  const int j = shift(i, kFwdX[d], kFwdY[d], nx, ny);
  const SiteF si = site_factors(L.n(p, 0, i), L.n(p, 1, i), gutz);
  const SiteF sj = site_factors(L.n(p, 0, j), L.n(p, 1, j), gutz);
  double sn, cs;
  sincos(phi[d * N + i], &sn, &cs);
  const Cplx dt = cx(-tamp * sn, tamp * cs);  // d/dphi of t e^{i phi}
  double g = 0.0;
  for (int s = 0; s < 2; ++s) {
    const double gg = si.gt[s] * sj.gt[s];
    const Cplx gT = L.chi(gf, s, d, i);
    // Re(conj(gT) dT), dT = -gg dt
    g += -gg * (gT.re * dt.re + gT.im * dt.im);
    const double de2 = 2.0 * cmul(dt, L.chi(p, s, d, i)).re;
    for (int sp = 0; sp < 2; ++sp) {
      g += L.n(gf, sp, i) * (-si.dgt[s][sp] * sj.gt[s] * de2);
      g += L.n(gf, sp, j) * (-sj.dgt[s][sp] * si.gt[s] * de2);
    }
  }
  out[d * N + i] = g;
}

}  // namespace

cudaError_t launch_phi_grad(const kpm_model& m, const double* phi, const double* params, const double* grad_fields,
                            double* grad_phi, cudaStream_t s) {
  const int N = m.nx * m.ny;
  phi_grad_kernel<<<(4 * N + 127) / 128, 128, 0, s>>>(m, phi, params, grad_fields, grad_phi);
  return cudaGetLastError();
}

int reduce_scratch_doubles(int64_t) { return 2 * kRedGrid + 16; }

cudaError_t launch_peierls(const kpm_model& m, double* phi, cudaStream_t s) {
  const int N = m.nx * m.ny;
  peierls_kernel<<<(N + 255) / 256, 256, 0, s>>>(m, phi);
  return cudaGetLastError();
}

cudaError_t launch_fields(const kpm_model& m, const double* phi, const double* params, double mu,
                          double* fields, double* wsite, cudaStream_t s) {
  const int N = m.nx * m.ny;
  fields_kernel<<<(N + 127) / 128, 128, 0, s>>>(m, phi, params, mu, fields, wsite);
  return cudaGetLastError();
}

cudaError_t launch_sum(const double* x, int64_t n, double* out, double* red, cudaStream_t s) {
  const int g = grid_for(n);
  reduce_partial<0><<<g, kRedBlock, 0, s>>>(x, n, red);
  reduce_final<0><<<1, kRedBlock, 0, s>>>(red, g, out, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_shift_eps(int N, double* fields, const double* mu_eff, double* mean_scratch, double* mu_out,
                             double* red, cudaStream_t s) {
  cudaError_t err = launch_sum(fields, 2 * (int64_t)N, mean_scratch, red, s);
  if (err != cudaSuccess) return err;
  shift_eps_kernel<<<grid_for(2 * (int64_t)N), kRedBlock, 0, s>>>(N, fields, mean_scratch, mu_eff, mu_out);
  return cudaGetLastError();
}

cudaError_t launch_gershgorin(const kpm_model& m, const double* fields, double margin, double* ab, double* red,
                              cudaStream_t s, int symmetric) {
  const int N = m.nx * m.ny;
  const int g = grid_for(N);
  gershgorin_partial<<<g, kRedBlock, 0, s>>>(m, fields, red);
  gershgorin_final<<<1, kRedBlock, 0, s>>>(red, g, margin, symmetric, ab);
  return cudaGetLastError();
}

__global__ void ph_asym_final(const double* __restrict__ part, int n, double* __restrict__ out) {
  double dev = 0.0, mag = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    dev = fmax(dev, part[2 * k]);
    mag = fmax(mag, part[2 * k + 1]);
  }
  dev = block_reduce<1>(dev);
  mag = block_reduce<1>(mag);
  if (threadIdx.x == 0) {
    out[0] = dev;
    out[1] = mag;
  }
}

cudaError_t launch_ph_asym(const kpm_model& m, const double* fields, double* out2, double* red, cudaStream_t s) {
  const int N = m.nx * m.ny;
  const int g = grid_for(N);
  ph_asym_partial<<<g, kRedBlock, 0, s>>>(m, fields, red);
  ph_asym_final<<<1, kRedBlock, 0, s>>>(red, g, out2);
  return cudaGetLastError();
}

// T > 0: c_m = (1/K) sum_k f(x_k) cos(m th_k), th_k = pi (k + 1/2)/K, x_k =
// cos th_k, K = 4 M (Chebyshev-Gauss quadrature, App. B) for the Fermi
// function f of eps = a x + b and for G = g(eps)/a, g(eps) = -T log(1 + e^{-eps/T});
// one block per m, the cosine argument reduced exactly as m (2k+1) mod 4K.
__global__ void coefficients_T_kernel(int M, const double* __restrict__ ab, double T, double* __restrict__ am,
                                      double* __restrict__ ao, int half) {
  const int m = blockIdx.x;
  const double a = ab[0], b = ab[1];
  const int64_t K = 4 * (int64_t)M;
  double sf = 0.0, sg = 0.0;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
    const double x = cospi((double)(2 * k + 1) / (double)(2 * K));
    const double e = a * x + b;
    const double f = 0.5 * (1.0 - tanh(0.5 * e / T));
    const double z = -e / T;  // softplus(z) = log(1 + e^z), evaluated without overflow
    const double sp = z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
    const double g = -T * sp / a;
    const int64_t n = ((int64_t)m * (2 * k + 1)) % (4 * K);
    const double c = cospi((double)n / (double)(2 * K));
    sf += f * c;
    sg += g * c;
  }
  sf = block_reduce<0>(sf);
  sg = block_reduce<0>(sg);
  if (threadIdx.x == 0) {
    const double q = kPi / (M + 1);
    const double gm = ((M - m + 1) * cos(q * m) + sin(q * m) * cos(q) / sin(q)) / (M + 1);
    const double w = m == 0 ? 1.0 : 2.0;
    am[m] = w * gm * sf / (double)K;
    const double o = w * gm * sg / (double)K;
    ao[m] = half ? ((m & 1) ? 0.0 : 2.0 * o) : o;
  }
}

// Vortex-profile order parameters (Eqs. giDelta, gm): the physical pairing
// Delta_i = 1/8 sum_{sigma,tau} g^t_i,sigma g^t_{i+tau},sigma (-1)^{tau_y}
// Delta_{i,i+tau,sigma} e^{i phi_{i,i+tau}} (Delta_up = F_ij, Delta_dn = F_ji; the
// bond phase sign makes Delta_i a pair at site i under gauge changes) and
// M_i = (-1)^{x+y} g^xy_i/4 sum_tau sqrt(R_{i,i+tau}) m_i (R = g^z/g^xy).
__global__ void order_parameters_kernel(kpm_model m, const double* __restrict__ phi, const double* __restrict__ p,
                                        double* __restrict__ delta_out, double* __restrict__ mag_out) {
  const int nx = m.nx, ny = m.ny, N = nx * ny;
  const Layout L{N};
  const bool gutz = m.gutzwiller != 0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const SiteF si = site_factors(L.n(p, 0, i), L.n(p, 1, i), gutz);
  Cplx dsum = cx(0.0, 0.0);
  double rsum = 0.0;
  for (int e = 0; e < 4; ++e) {
    const int j = shift(i, kNnX[e], kNnY[e], nx, ny);
    const SiteF sj = site_factors(L.n(p, 0, j), L.n(p, 1, j), gutz);
    // phase of the bond i -> j: forward +x/+y stored at i, -x/-y minus the forward phase at j
    const double ph = e < 2 ? phi[e * N + i] : -phi[(e - 2) * N + j];
    double sn, cs;
    sincos(ph, &sn, &cs);
    const Cplx term = cadd(cscale(L.F(p, e, i), si.gt[0] * sj.gt[0]), cscale(L.F(p, (e + 2) & 3, j), si.gt[1] * sj.gt[1]));
    dsum = cadd(dsum, cscale(cmul(term, cx(cs, sn)), e == 1 || e == 3 ? -1.0 : 1.0));
    // exchange ratio R of the bond (stored at its forward end)
    const int d = e & 1;
    const int a = e < 2 ? i : j, b = e < 2 ? j : i;
    const SiteF& sa = e < 2 ? si : sj;
    const SiteF& sb = e < 2 ? sj : si;
    const BondX bx = bond_exchange(sa, sb, L.chi(p, 0, d, a), L.chi(p, 1, d, a), L.F(p, d, a), L.F(p, d + 2, b),
                                   m.J, gutz);
    rsum += sqrt(bx.R);
  }
  delta_out[2 * i] = dsum.re / 8.0;
  delta_out[2 * i + 1] = dsum.im / 8.0;
  const int x = i % nx, y = i / nx;
  mag_out[i] = ((x + y) & 1 ? -1.0 : 1.0) * si.gxy / 4.0 * rsum * si.m;
}

cudaError_t launch_order_parameters(const kpm_model& m, const double* phi, const double* params, double* delta_out,
                                    double* mag_out, cudaStream_t s) {
  const int N = m.nx * m.ny;
  order_parameters_kernel<<<(N + 127) / 128, 128, 0, s>>>(m, phi, params, delta_out, mag_out);
  return cudaGetLastError();
}

__global__ void gt_weights_kernel(kpm_model m, const double* __restrict__ params, double* __restrict__ w) {
  const int N = m.nx * m.ny;
  const Layout L{N};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const SiteF f = site_factors(L.n(params, 0, i), L.n(params, 1, i), m.gutzwiller != 0);
  w[i] = f.gt[0] * f.gt[0];
  w[N + i] = f.gt[1] * f.gt[1];
}

cudaError_t launch_gt_weights(const kpm_model& m, const double* params, double* w, cudaStream_t s) {
  const int N = m.nx * m.ny;
  gt_weights_kernel<<<(N + 127) / 128, 128, 0, s>>>(m, params, w);
  return cudaGetLastError();
}

cudaError_t launch_coefficients(int M, const double* ab, double* am, double* ao, cudaStream_t s, int half,
                                double temperature) {
  if (temperature > 0.0)
    coefficients_T_kernel<<<M, kRedBlock, 0, s>>>(M, ab, temperature, am, ao, half);
  else
    coefficients_kernel<<<(M + 255) / 256, 256, 0, s>>>(M, ab, am, ao, half);
  return cudaGetLastError();
}

cudaError_t launch_scale_table_f32(const kpm_model& m, const double* fields, const double* ab, float2* table,
                                   cudaStream_t s) {
  const int N = m.nx * m.ny;
  scale_table_kernel<float2><<<(N + 127) / 128, 128, 0, s>>>(m, fields, ab, table);
  return cudaGetLastError();
}

cudaError_t launch_scale_table_df(const kpm_model& m, const double* fields, const double* ab, float4* table,
                                  cudaStream_t s) {
  const int N = m.nx * m.ny;
  scale_table_kernel<float4><<<(N + 127) / 128, 128, 0, s>>>(m, fields, ab, table);
  return cudaGetLastError();
}

cudaError_t launch_scale_table_f64(const kpm_model& m, const double* fields, const double* ab, double2* table,
                                   cudaStream_t s) {
  const int N = m.nx * m.ny;
  scale_table_kernel<double2><<<(N + 127) / 128, 128, 0, s>>>(m, fields, ab, table);
  return cudaGetLastError();
}

cudaError_t launch_assemble(int nx, int ny, const double2* acc, const double* ab, double* obs, double* omega,
                            double* red, cudaStream_t s, int half, int sb, int se) {
  const int g = grid_for(nx * ny);
  assemble_kernel<<<g, kRedBlock, 0, s>>>(nx, ny, acc, obs, red, half, sb, se < 0 ? nx * ny : se);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess || omega == nullptr) return err;
  // omega = a * sum Re acc[J][9]; a read on the device
  reduce_final<0><<<1, kRedBlock, 0, s>>>(red, g, omega, ab);
  return cudaGetLastError();
}

cudaError_t launch_update(int N, double* params, double* obs, double* mu_eff, const kpm_rmft_opts& o,
                          double* stats, double* red, cudaStream_t s, double* rec, const double* snap,
                          const AndersonState* an) {
  double* nsum = red + 2 * kRedGrid + 8;
  cudaError_t err = launch_sum(obs, 2 * (int64_t)N, nsum, red, s);
  if (err != cudaSuccess) return err;
  if (an == nullptr || an->m < 1) {
    const int g = grid_for(25 * (int64_t)N);
    update_kernel<<<g, kRedBlock, 0, s>>>(N, params, obs, nsum, o, red, rec);
    update_final<<<1, kRedBlock, 0, s>>>(red, g, N, nsum, o, mu_eff, stats, rec, snap);
    return cudaGetLastError();
  }
  const int m = an->m;
  const int64_t L = 26 * (int64_t)N + 1;
  const int g = grid_for(25 * (int64_t)N + 1);
  anderson_resid_kernel<<<g, kRedBlock, 0, s>>>(N, params, obs, nsum, mu_eff, o, m, an->xprev, an->fprev, an->fcur,
                                                an->dX, an->dF, red, rec);
  const int pairs = m * (m + 3) / 2;  // (a, b) with a <= b < m, and (a, f)
  anderson_gram_kernel<<<dim3(pairs, kAndChunks), kRedBlock, 0, s>>>(L, m, an->dF, an->fcur, an->gpart, rec);
  anderson_solve_kernel<<<1, 32, 0, s>>>(m, an->gpart, an->gamma, rec);
  anderson_apply_kernel<<<grid_for(L), kRedBlock, 0, s>>>(N, params, mu_eff, m, an->fcur, an->dX, an->dF, an->gamma,
                                                          rec);
  anderson_final<<<1, kRedBlock, 0, s>>>(red, g, N, nsum, o, stats, rec, snap);
  return cudaGetLastError();
}

size_t anderson_doubles(int N, int m) {
  const size_t L = 26 * (size_t)N + 1;
  return (2 * (size_t)m + 3) * L + (size_t)(m * (m + 3) / 2) * kAndChunks + 16;
}

AndersonState anderson_state(int N, int m, double* base) {
  const size_t L = 26 * (size_t)N + 1;
  AndersonState a;
  a.m = m;
  a.dX = base;
  a.dF = base + (size_t)m * L;
  a.xprev = base + 2 * (size_t)m * L;
  a.fprev = a.xprev + L;
  a.fcur = a.fprev + L;
  a.gpart = a.fcur + L;
  a.gamma = a.gpart + (size_t)(m * (m + 3) / 2) * kAndChunks;
  return a;
}

}  // namespace kpm
