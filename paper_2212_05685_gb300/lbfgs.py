"""Gradient-based RMFT: L-BFGS over the effective fields, driven by kpm_backward.

Parametrise the state by the effective fields theta = (eps, T, D) of the
Nambu matrix (App. B) and minimise the self-consistency residual in field
space,

    R(theta) = 1/2 || g(fields(O(theta))) - g(theta) ||^2,

where O(theta) are the KPM observables of h(theta), fields(O) = dW/d(n, chi,
F*) the effective fields of App. A at those observables (kpm_build_H), and
g(x) = (eps, 2 conj T, 2 D) their real-layout dual (g(fields(O)) is the real
gradient of W).  R vanishes exactly at the fixed point of the RMFT loop.
With r = g(fields(O)) - g(theta),

    dR/dtheta = J^T (H_W r) - D_g r,

J = dO/dtheta applied transposed by one adjoint pass (kpm_backward), H_W the
(symmetric) Hessian of W in the real layout applied to r by a central
difference of two kpm_build_H calls, D_g = dg/dtheta (diagonal 1, 2).
The energy W(O(theta)) itself is not used: the smoothed occupations of a
truncated, damped series are not a Slater projector, and W is unbounded
below over such states.  The chemical potential is held fixed; (a, b) are
held at the starting Hamiltonian's bounds widened by `widen`.

All KPM work runs in the library's kernels; this module is the optimiser
(limited-memory BFGS on the GPU-resident field vector) around them.
"""
from __future__ import annotations

import torch

from . import kpm


def _dual(x, N):
    """g(x) = (eps, 2 conj T, 2 D) in the real 26N layout."""
    g = x.clone()
    g[2 * N:18 * N] *= 2.0
    g[2 * N + 1:18 * N:2] *= -1.0
    g[18 * N:] *= 2.0
    return g


class FieldProblem:
    def __init__(self, ctx, model, opts, phi, mu, theta0, widen=0.05):
        self.ctx, self.model, self.opts, self.phi, self.mu = ctx, model, opts, phi, float(mu)
        self.last_residual = None
        self.N = model.nx * model.ny
        dev = theta0.device
        ab = torch.empty(2, dtype=torch.float64, device=dev)
        kpm.kpm_bounds(ctx, model, theta0, 0.01 + widen, ab)
        self.ab = ab
        self.obs = torch.empty(26 * self.N, dtype=torch.float64, device=dev)
        self.omega = torch.empty(1, dtype=torch.float64, device=dev)
        self.fW = torch.empty(26 * self.N, dtype=torch.float64, device=dev)
        self.w = torch.empty(1, dtype=torch.float64, device=dev)
        self.grad = torch.empty(26 * self.N, dtype=torch.float64, device=dev)
        self.passes = 0

    def value_and_grad(self, theta):
        N = self.N
        kpm.kpm_observables(self.ctx, self.model, self.opts, theta, self.ab, self.obs, self.omega)
        kpm.kpm_build_H(self.ctx, self.model, self.phi, self.obs, self.mu, self.fW, self.w)
        r = _dual(self.fW, N) - _dual(theta, N)
        # H_W r by a central difference of the fields along r (in the observable space)
        t = 1e-6 / max(float(r.abs().max()), 1e-30)
        fp = torch.empty_like(self.fW)
        fm = torch.empty_like(self.fW)
        kpm.kpm_build_H(self.ctx, self.model, self.phi, self.obs + t * r, self.mu, fp)
        kpm.kpm_build_H(self.ctx, self.model, self.phi, self.obs - t * r, self.mu, fm)
        hr = (_dual(fp, N) - _dual(fm, N)) / (2.0 * t)
        kpm.kpm_backward(self.ctx, self.model, self.opts, theta, self.ab, hr, 0.0, self.grad)
        self.passes += 2
        grad = self.grad - _dual(r, N)
        self.last_residual = float(r.abs().max())
        return 0.5 * torch.dot(r, r), grad

    def residual(self, theta):
        """max |g(fields(O(theta))) - g(theta)| without the gradient (one pass)."""
        N = self.N
        kpm.kpm_observables(self.ctx, self.model, self.opts, theta, self.ab, self.obs, self.omega)
        kpm.kpm_build_H(self.ctx, self.model, self.phi, self.obs, self.mu, self.fW, self.w)
        self.passes += 1
        return float((_dual(self.fW, N) - _dual(theta, N)).abs().max())

    def physical(self):
        """Every site density of the last evaluation lies in (0, 1)."""
        N = self.N
        n = self.obs[:N] + self.obs[N:2 * N]
        return bool(((n > 0.0) & (n < 1.0)).all())


def _inside(ctx, model, theta, ab_fixed, scratch):
    """True when theta's Gershgorin interval lies inside the fixed rescaling
    interval [b - a, b + a] (so the Chebyshev series stays bounded)."""
    kpm.kpm_bounds(ctx, model, theta, 0.0, scratch)
    a1, b1 = scratch.tolist()
    a0, b0 = ab_fixed.tolist()
    return (b1 - a1 >= b0 - a0) and (b1 + a1 <= b0 + a0)


def rmft_lbfgs(ctx, model, opts, phi, params0, mu, max_iter=200, tol=1e-9, history=20, widen=0.05, trace=None):
    """Minimise Phi over the fields starting from the fields of params0.

    Limited-memory BFGS (two-loop recursion) with an Armijo backtracking line
    search that rejects trial fields outside the fixed rescaling interval, with
    non-finite values, or with a site density outside (0, 1).  Stops when the
    largest field-space residual component is below tol.  Returns (theta, obs, info) with info =
    {iterations, passes, phi, grad_max, field_residual}, field_residual =
    max |fields(O(theta)) - theta|.  trace: optional list that receives
    (KPM passes so far, field residual) after every accepted step.
    """
    N = model.nx * model.ny
    x = torch.empty(26 * N, dtype=torch.float64, device=params0.device)
    kpm.kpm_build_H(ctx, model, phi, params0, mu, x)
    prob = FieldProblem(ctx, model, opts, phi, mu, x, widen)
    scratch = torch.empty(2, dtype=torch.float64, device=x.device)
    f, g = prob.value_and_grad(x)
    f = float(f)
    S, Y = [], []
    it = 0
    for it in range(1, max_iter + 1):
        if prob.last_residual < tol:
            break
        # two-loop recursion for d = -H g
        q = -g.clone()
        alphas = []
        for s_k, y_k in reversed(list(zip(S, Y))):
            rho = 1.0 / float(torch.dot(y_k, s_k))
            a_k = rho * float(torch.dot(s_k, q))
            alphas.append((rho, a_k))
            q -= a_k * y_k
        if S:
            q *= float(torch.dot(S[-1], Y[-1])) / float(torch.dot(Y[-1], Y[-1]))
        else:
            q *= 1e-2 / max(float(g.abs().max()), 1e-30)
        for (s_k, y_k), (rho, a_k) in zip(zip(S, Y), reversed(alphas)):
            b_k = rho * float(torch.dot(y_k, q))
            q += (a_k - b_k) * s_k
        slope = float(torch.dot(g, q))
        if slope >= 0.0:  # not a descent direction: restart from steepest descent
            S, Y = [], []
            q = -g * (1e-2 / max(float(g.abs().max()), 1e-30))
            slope = float(torch.dot(g, q))
        step, accepted = 1.0, False
        while step > 1e-12:
            xn = x + step * q
            if _inside(ctx, model, xn, prob.ab, scratch):
                fn, gn = prob.value_and_grad(xn)
                fn = float(fn)
                if (fn == fn and abs(fn) < 1e300 and bool(torch.isfinite(gn).all()) and prob.physical()
                        and fn <= f + 1e-4 * step * slope):
                    accepted = True
                    break
            step *= 0.5
        if not accepted:
            break
        s_k, y_k = xn - x, gn - g
        if float(torch.dot(s_k, y_k)) > 1e-16 * float(torch.dot(y_k, y_k)):
            S.append(s_k)
            Y.append(y_k)
            if len(S) > history:
                S.pop(0)
                Y.pop(0)
        x, f, g = xn, fn, gn
        if trace is not None:
            trace.append((prob.passes, prob.last_residual))
    prob.value_and_grad(x)
    info = {"iterations": it, "passes": prob.passes, "objective": f, "grad_max": float(g.abs().max()),
            "field_residual": prob.last_residual}
    return x, prob.obs.clone(), info
