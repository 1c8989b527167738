"""Reverse-mode gradients of the KPM observables (oracle; test infrastructure only).

App. B, Eqs. dFdH, dalphadH: with alpha_m = T_m(h~) r, the derivative of any
linear functional of the alpha_m with respect to h~ follows from a second,
backward recursion for beta_m = dE/dalpha_{m+1} with the same matrix, and
dE/dh_IJ = beta_0,I alpha_0,J + 2 sum_m beta_m,I alpha_m,J.

Conventions.  A real loss L of complex quantities z uses the gradient
g = dL/dRe z + i dL/dIm z (so dL = Re(conj(g) dz)); for real quantities g is
the ordinary derivative.  Upstream gradients come in the order-parameter
layout (26 N) for (n, chi, F) and a scalar for Omega; results come in the
field layout for (eps, T, D) = the effective fields, plus 4 N for the Peierls
phases.  The rescaling (a, b) is held fixed (it is a Gershgorin bound, not a
smooth function of h).

Three routes:
  vjp_dense      Daleckii-Krein: df(h)[E] = U (Phi o U^dag E U) U^dag with the
                 divided differences Phi of the damped series (exact for the
                 matrix polynomial; independent of the recursion)
  vjp_recursion  the backward recursion of App. B on unit start vectors
  field chain    the Nambu matrix entries as functions of (eps, T, D) and of
                 the Peierls phases (App. A, B)
"""
from __future__ import annotations

import numpy as np

from .bdg import dense
from .kpm import cheb_eval, coefficients
from .lattice import NN4
from .rmft import join, site_factors, split


# ----------------------------------------------------------------------------- seed matrix

def seed_matrix(model, g_obs, D):
    """W with dL = Re sum_KJ conj(W_KJ) dF_KJ for L = <g_obs, obs(F)> (readings N2, N3)."""
    N = model.N
    gn, gc, gF = split(g_obs, N)
    W = np.zeros((D, D), dtype=np.complex128)
    i = np.arange(N)
    np.add.at(W, (2 * i, 2 * i), gn[0])
    np.add.at(W, (2 * i + 1, 2 * i + 1), -gn[1])
    for d in range(4):
        j = model.fwd[d]
        np.add.at(W, (2 * j, 2 * i), gc[0, d])
        np.add.at(W, (2 * j + 1, 2 * i + 1), -np.conj(gc[1, d]))
    for e in range(4):
        j = model.nn4[e]
        np.add.at(W, (2 * j + 1, 2 * i), -np.conj(gF[e]))
    return W


def loss(model, obs, g_obs, omega, g_omega):
    """L = <g_obs, obs> + g_omega * Omega in the real-inner-product convention."""
    return float(np.sum(np.asarray(g_obs) * np.asarray(obs)) + g_omega * omega)


# ----------------------------------------------------------------------------- gradient in h~

def _divided_differences(fx, fpx, x):
    dx = x[:, None] - x[None, :]
    same = np.abs(dx) < 1e-12
    with np.errstate(divide="ignore", invalid="ignore"):
        Phi = (fx[:, None] - fx[None, :]) / np.where(same, 1.0, dx)
    return np.where(same, 0.5 * (fpx[:, None] + fpx[None, :]), Phi)


def _cheb_deriv_eval(a, x):
    """d/dx sum_m a_m T_m(x) = sum_m a_m m U_{m-1}(x)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    if len(a) < 2:
        return out
    u0 = np.ones_like(x)          # U_0
    out = out + a[1] * 1 * u0
    if len(a) < 3:
        return out
    u1 = 2.0 * x                  # U_1
    out = out + a[2] * 2 * u1
    for m in range(3, len(a)):
        u0, u1 = u1, 2.0 * x * u1 - u0
        out = out + a[m] * m * u1
    return out


def grad_htilde_dense(h, a, b, M, W, g_omega):
    """G with dL = Re sum conj(G_IK) dh~_IK (Daleckii-Krein)."""
    D = h.shape[0]
    E, U = np.linalg.eigh(h)
    x = (E - b) / a
    am, ao = coefficients(M, a, b)
    Phi = _divided_differences(cheb_eval(am, x), _cheb_deriv_eval(am, x), x)
    Wt = U.conj().T @ W @ U
    G = U @ (Phi * Wt) @ U.conj().T
    # Omega = a tr G_M(h~): d Omega = a tr(G_M'(h~) dh~)  ->  gradient a G_M'(h~)^dag
    gp = _cheb_deriv_eval(ao, x)
    G = G + g_omega * a * (U * gp) @ U.conj().T
    return G


def grad_htilde_recursion(hcsr, a, b, M, W, g_omega, cols=None):
    """Backward recursion of App. B on unit columns: returns the dense G (D x D).

    For column J: alpha_0 = e_J, alpha_1 = h~ alpha_0, alpha_{m+1} = 2 h~ alpha_m
    - alpha_{m-1}; L_J = Re sum_m c_m^dag alpha_m with c_m = a_m W[:, J] +
    a g_Omega a^Omega_m e_J; lambda_m = c_m + 2 h~ lambda_{m+1} - lambda_{m+2}
    (lambda_M = lambda_{M+1} = 0); G += lambda_1 alpha_0^dag + 2 sum_{m>=2}
    lambda_m alpha_{m-1}^dag.
    """
    import scipy.sparse as sp
    D = hcsr.shape[0]
    ht = ((hcsr - b * sp.identity(D, dtype=np.complex128, format="csr")) / a).toarray()
    am, ao = coefficients(M, a, b)
    cols = np.arange(D) if cols is None else np.asarray(cols)
    G = np.zeros((D, D), dtype=np.complex128)
    for J in cols:
        alpha = np.zeros((M, D), dtype=np.complex128)
        alpha[0, J] = 1.0
        if M > 1:
            alpha[1] = ht @ alpha[0]
        for m in range(2, M):
            alpha[m] = 2.0 * ht @ alpha[m - 1] - alpha[m - 2]
        w = W[:, J]
        lam_next = np.zeros(D, dtype=np.complex128)   # lambda_{m+1}
        lam_next2 = np.zeros(D, dtype=np.complex128)  # lambda_{m+2}
        for m in range(M - 1, 0, -1):
            c = am[m] * w
            c = c.copy()
            c[J] += a * g_omega * ao[m]
            lam = c + 2.0 * ht @ lam_next - lam_next2
            G += (1.0 if m == 1 else 2.0) * np.outer(lam, np.conj(alpha[m - 1]))
            lam_next2, lam_next = lam_next, lam
    return G


# ----------------------------------------------------------------------------- chain to fields and phases

def field_grad_from_G(model, G, a):
    """dL/d(eps, T, D) from the h~ gradient G, h~ = (h - b)/a with the Nambu
    entries of bdg.py: (eps_up, -eps_dn) diagonals, T_up and -conj(T_dn) hops,
    -D pairings, and Hermitian conjugates."""
    N = model.N
    i = np.arange(N)
    Gh = G / a
    eps = np.zeros((2, N))
    T = np.zeros((2, 4, N), dtype=np.complex128)
    Dg = np.zeros((4, N), dtype=np.complex128)
    eps[0] = Gh[2 * i, 2 * i].real
    eps[1] = -Gh[2 * i + 1, 2 * i + 1].real
    for d in range(4):
        j = model.fwd[d]
        T[0, d] = Gh[2 * i, 2 * j] + np.conj(Gh[2 * j, 2 * i])
        T[1, d] = -(np.conj(Gh[2 * i + 1, 2 * j + 1]) + Gh[2 * j + 1, 2 * i + 1])
    for e in range(4):
        j = model.nn4[e]
        Dg[e] = -(Gh[2 * i, 2 * j + 1] + np.conj(Gh[2 * j + 1, 2 * i]))
    return join(eps, T, Dg)


def vjp_dense(model, fld, a, b, M, g_obs, g_omega):
    h = dense(model, fld)
    W = seed_matrix(model, g_obs, h.shape[0])
    return field_grad_from_G(model, grad_htilde_dense(h, a, b, M, W, g_omega), a)


def vjp_recursion(model, fld, a, b, M, g_obs, g_omega):
    from .bdg import csr
    h = csr(model, fld)
    W = seed_matrix(model, g_obs, h.shape[0])
    return field_grad_from_G(model, grad_htilde_recursion(h, a, b, M, W, g_omega), a)


def phi_grad(model, params, g_fields):
    """dL/dphi through the fields (App. A): T_{ij s} contains -g^t_{ij s} t_ij
    e^{i phi_ij}, and eps_{i s} contains -sum dg^t/dn * g^t * 2 Re(t_ij chi_ij s)
    at both ends of each bond."""
    N = model.N
    n, chi, F = split(params, N)
    sf = site_factors(n, model.gutzwiller)
    geps, gT, _ = split(g_fields, N)
    tamp = np.array([model.t, model.t, model.tp, model.tp])
    out = np.zeros((4, N))
    for d in range(4):
        j = model.fwd[d]
        t_ij = tamp[d] * np.exp(1j * model.phi[d])
        dt = 1j * t_ij  # d t_ij / d phi
        for s in range(2):
            gg = sf["gt"][s] * sf["gt"][s][j]
            dT = -gg * dt
            out[d] += (np.conj(gT[s, d]) * dT).real
            de2 = 2.0 * (dt * chi[s, d]).real
            for sp in range(2):
                out[d] += geps[sp] * (-sf["dgt"][s, sp] * sf["gt"][s][j] * de2)
                out[d] += geps[sp][j] * (-sf["dgt"][s, sp][j] * sf["gt"][s] * de2)
    return out.reshape(-1)
