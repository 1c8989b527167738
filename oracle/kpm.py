"""Kernel polynomial method: coefficients and three density-matrix routes (oracle).

TEST INFRASTRUCTURE ONLY.  Follows App. B of arXiv:2212.05685.

Rescaling: h~ = (h - b)/a with (a, b) from the Gershgorin bounds (bdg.py).

Coefficients.  For a function f on [-1, 1] its Chebyshev expansion is
f(x) = sum_m (2 - delta_m0) c_m T_m(x) with c_m = int f T_m /(pi sqrt(1-x^2)) dx;
the damped series multiplies term m by the Jackson factor g_m (reading K2):
    g_m = [(M-m+1) cos(pi m/(M+1)) + sin(pi m/(M+1)) cot(pi/(M+1))] / (M+1).
At T = 0 the occupation is the step theta(x0 - x) with x0 = -b/a (BdG energy
0, reading K3), theta0 = arccos x0:
    c_0 = 1 - theta0/pi,   c_m = -sin(m theta0)/(m pi).
The grand-potential function of Eq. F_KPM at T -> 0 is min(eps, 0) = a min(x - x0, 0):
    c^Omega_m = (1/pi) [ (S_{m+1} + S_{m-1})/2 - x0 S_m ],
    S_0 = pi - theta0, S_k = -sin(k theta0)/k.
`chebyshev_gauss` evaluates c_m by Chebyshev-Gauss quadrature, the route the
paper names for C_m; the tests compare the two.

Density matrix.  rho_IJ = <d^dagger_I d_J> = f(h)_JI, so column J of f(h)
holds the correlations of d_J with every d_K.  Three routes to f(h):
  O0  exact ground state: U theta(-E) U^dagger, weight 1/2 at E = 0;
  O1  spectral KPM: U F_M((E - b)/a) U^dagger, F_M the damped step series;
  O2  naive KPM: the recursion of Eq. alpha on unit start vectors e_J
      (alpha_0 = e_J, alpha_1 = h~ e_J, alpha_m = 2 h~ alpha_{m-1} - alpha_{m-2})
      summing a_m alpha_m; all D columns, i.e. the exact trace (reading K5).
O1 and O2 agree to rounding; O0 is their M -> infinity limit.
"""
from __future__ import annotations

import numpy as np

from .rmft import join


def jackson(M):
    m = np.arange(M, dtype=np.float64)
    q = np.pi / (M + 1)
    return ((M - m + 1) * np.cos(q * m) + np.sin(q * m) / np.tan(q)) / (M + 1)


def step_coeffs(M, x0):
    th = np.arccos(np.clip(x0, -1.0, 1.0))
    m = np.arange(M, dtype=np.float64)
    c = np.empty(M)
    c[0] = 1.0 - th / np.pi
    c[1:] = -np.sin(m[1:] * th) / (m[1:] * np.pi)
    return c


def omega_coeffs(M, x0):
    th = np.arccos(np.clip(x0, -1.0, 1.0))

    def S(k):
        k = np.abs(np.asarray(k, dtype=np.float64))
        safe = np.where(k == 0, 1.0, k)
        return np.where(k == 0, np.pi - th, -np.sin(k * th) / safe)

    m = np.arange(M, dtype=np.float64)
    return (0.5 * (S(m + 1) + S(m - 1)) - x0 * S(m)) / np.pi


def chebyshev_gauss(f, M, K):
    """c_m = (1/K) sum_k f(cos th_k) cos(m th_k), th_k = pi (k + 1/2)/K."""
    th = np.pi * (np.arange(K) + 0.5) / K
    fx = f(np.cos(th))
    m = np.arange(M)[:, None]
    return (np.cos(m * th[None, :]) @ fx) / K


def series(c, M, damp=True):
    """a_m = (2 - delta_m0) g_m c_m."""
    g = jackson(M) if damp else np.ones(M)
    a = 2.0 * g * c[:M]
    a[0] *= 0.5
    return a


def cheb_eval(a, x):
    """sum_m a_m T_m(x) by the three-term recursion (|x| <= 1)."""
    x = np.asarray(x, dtype=np.float64)
    t0 = np.ones_like(x)
    out = a[0] * t0
    if len(a) == 1:
        return out
    t1 = x.copy()
    out = out + a[1] * t1
    for m in range(2, len(a)):
        t0, t1 = t1, 2.0 * x * t1 - t0
        out = out + a[m] * t1
    return out


def fermi(eps, T):
    """Occupation 1 / (1 + e^{eps/T}) (T > 0)."""
    return 0.5 * (1.0 - np.tanh(0.5 * np.asarray(eps, dtype=np.float64) / T))


def grand(eps, T):
    """Grand-potential function -T log(1 + e^{-eps/T}); min(eps, 0) as T -> 0."""
    eps = np.asarray(eps, dtype=np.float64)
    return -T * np.logaddexp(0.0, -eps / T)


def coefficients(M, a, b, T=0.0, K=None):
    """(a_m of the occupation, a^Omega_m of the grand-potential function) for
    bounds (a, b): at T = 0 the step theta(x0 - x) and min(x - x0, 0) in closed
    form (reading K3); at T > 0 (Eq. F_KPM with f = -T log(1 + e^{-(eps)/T}),
    eps = a x + b) both by Chebyshev-Gauss quadrature with K = 4M nodes, the
    route App. B names for C_m."""
    if T <= 0.0:
        x0 = -b / a
        return series(step_coeffs(M, x0), M), series(omega_coeffs(M, x0), M)
    K = 4 * M if K is None else K
    c = chebyshev_gauss(lambda x: fermi(a * x + b, T), M, K)
    co = chebyshev_gauss(lambda x: grand(a * x + b, T) / a, M, K)
    return series(c, M), series(co, M)


# ----------------------------------------------------------------------------- density matrices

def f_ed(h, T=0.0):
    """O0: exact occupation U f(E) U^dagger and Omega = sum_n g(E_n): at T = 0
    the step (ties at E = 0 weigh 1/2) and min(E, 0); else Fermi and
    -T log(1 + e^{-E/T})."""
    E, U = np.linalg.eigh(h)
    if T > 0.0:
        return (U * fermi(E, T)) @ U.conj().T, float(np.sum(grand(E, T)))
    occ = np.where(E < 0, 1.0, np.where(E > 0, 0.0, 0.5))
    return (U * occ) @ U.conj().T, float(np.sum(np.minimum(E, 0.0)))


def f_spectral(h, a, b, M, T=0.0):
    """O1: U F_M((E - b)/a) U^dagger and Omega_M = a tr G_M(h~)."""
    E, U = np.linalg.eigh(h)
    x = (E - b) / a
    am, ao = coefficients(M, a, b, T)
    Fx = cheb_eval(am, x)
    Gx = cheb_eval(ao, x)
    return (U * Fx) @ U.conj().T, float(a * np.sum(Gx))


def f_naive(hcsr, a, b, M, cols=None, block=256):
    """O2: F_M(h~) e_J for the requested columns by the Chebyshev recursion.

    Returns (F, Omega_part): F[:, k] = F_M(h~) e_{cols[k]};
    Omega_part = a sum_{J in cols} sum_m a^Omega_m [T_m(h~) e_J]_J.
    """
    D = hcsr.shape[0]
    cols = np.arange(D) if cols is None else np.asarray(cols)
    import scipy.sparse as sp
    ht = (hcsr - b * sp.identity(D, dtype=np.complex128, format="csr")) / a
    am, ao = coefficients(M, a, b)
    out = np.zeros((D, len(cols)), dtype=np.complex128)
    om = 0.0
    for s in range(0, len(cols), block):
        cs = cols[s:s + block]
        V0 = np.zeros((D, len(cs)), dtype=np.complex128)
        V0[cs, np.arange(len(cs))] = 1.0
        acc = am[0] * V0
        omv = ao[0] * V0[cs, np.arange(len(cs))]
        if M > 1:
            V1 = ht @ V0
            acc = acc + am[1] * V1
            omv = omv + ao[1] * V1[cs, np.arange(len(cs))]
            for m in range(2, M):
                V0, V1 = V1, 2.0 * (ht @ V1) - V0
                acc = acc + am[m] * V1
                omv = omv + ao[m] * V1[cs, np.arange(len(cs))]
        out[:, s:s + len(cs)] = acc
        om += float(np.sum(omv.real))
    return out, a * om


# ----------------------------------------------------------------------------- observables

def observables(model, Fmat):
    """Order parameters from a full f(h) matrix (readings N2, N3)."""
    N = model.N
    i = np.arange(N)
    n = np.empty((2, N))
    n[0] = Fmat[2 * i, 2 * i].real
    n[1] = 1.0 - Fmat[2 * i + 1, 2 * i + 1].real
    chi = np.empty((2, 4, N), dtype=np.complex128)
    F = np.empty((4, N), dtype=np.complex128)
    for d in range(4):
        j = model.fwd[d]
        chi[0, d] = Fmat[2 * j, 2 * i]
        chi[1, d] = -np.conj(Fmat[2 * j + 1, 2 * i + 1])
    for e in range(4):
        j = model.nn4[e]
        F[e] = -np.conj(Fmat[2 * j + 1, 2 * i])
    return join(n, chi, F)


def observables_from_columns(model, cols_mat):
    """Same as `observables` when cols_mat holds all D columns of f(h)."""
    return observables(model, cols_mat)


def observables_at(model, Fc, cols, sites):
    """Order parameters of `sites` (readings N2, N3) from the columns of f(h)
    they need: Fc[:, k] is column cols[k]; every site j needs columns 2j and
    2j + 1.  Returns (n (2, k), chi (2, 4, k), F (4, k)) for the k sites, the
    same entries `observables` reads from a full matrix."""
    pos = {int(c): k for k, c in enumerate(cols)}
    sites = np.asarray(sites)
    n = np.empty((2, len(sites)))
    chi = np.empty((2, 4, len(sites)), dtype=np.complex128)
    F = np.empty((4, len(sites)), dtype=np.complex128)
    for k, i in enumerate(sites):
        c0, c1 = Fc[:, pos[2 * int(i)]], Fc[:, pos[2 * int(i) + 1]]
        n[0, k] = c0[2 * i].real
        n[1, k] = 1.0 - c1[2 * i + 1].real
        for d in range(4):
            j = model.fwd[d][i]
            chi[0, d, k] = c0[2 * j]
            chi[1, d, k] = -np.conj(c1[2 * j + 1])
        for e in range(4):
            j = model.nn4[e][i]
            F[e, k] = -np.conj(c0[2 * j + 1])
    return n, chi, F
