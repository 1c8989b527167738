"""Renormalised mean-field functional W and its effective fields (oracle).

TEST INFRASTRUCTURE ONLY.  Follows App. A of arXiv:2212.05685:

  g^t_{i s}   = sqrt( 2 delta (1-delta)/(1-delta^2+4m^2) * (1+delta+2 s m)/(1+delta-2 s m) )
  g^{s,xy}_i  = 2 (1-delta) / (1-delta^2+4m^2)
  g^{s,z}_ij  = g^{s,xy}_ij * [A - 4 m_i m_j X^2] / [A - 4 m_i m_j],
                A = 2(|Dbar|^2 - |chibar|^2)                  (reading W3)
  X_ij        = 1 + 12(1-delta_i)(1-delta_j)/sqrt(P_i P_j),  P = 1-delta^2+4m^2
  W           = <H_renorm> - mu (sum_i n_i - N_e)

with delta_i = 1 - n_{i up} - n_{i dn} and m_i = (n_{i up} - n_{i dn})/2.

<H_renorm> in a collinear Slater state, by Wick's theorem (reading W2):
  hopping  : - sum_{bonds, s} g^t_{ij s} (t_ij chi_{ij s} + c.c.)
  exchange : sum_{nn} J [ g^z (m_i m_j - 1/4 sum_s(|chi_s|^2 + |Delta_s|^2))
                          - g^xy Re(chi_up chi_dn^* + Delta_up^* Delta_dn) ]
with Delta_{ij up} = F_ij and Delta_{ij dn} = F_ji, F_ij = <c_{i up} c_{j dn}>.

Effective fields (Eqs. Tij, Dij, mu_i): T_{ij s} = dW/dchi_{ij s},
D_ij = dW/dF*_ij (Wirtinger derivatives), eps_{i s} = dW/dn_{i s}.
The function `fields` evaluates them analytically; the tests check them
against central finite differences of `energy_W`.

Both the order parameters and the fields use one flat float64 layout of
length 26N: [n or eps](2,N) | [chi or T](2,4,N) complex | [F or D](4,N) complex.
"""
from __future__ import annotations

import numpy as np

from .lattice import FWD, NN4, neighbour_table, peierls_phases

CLAMP = 1e-12


def split(p, N):
    p = np.ascontiguousarray(p, dtype=np.float64)
    a = p[0:2 * N].reshape(2, N)
    b = p[2 * N:18 * N].view(np.complex128).reshape(2, 4, N)
    c = p[18 * N:26 * N].view(np.complex128).reshape(4, N)
    return a, b, c


def join(a, b, c):
    N = np.shape(a)[1]
    out = np.empty(26 * N)
    out[0:2 * N] = np.asarray(a, dtype=np.float64).reshape(-1)
    out[2 * N:18 * N] = np.asarray(b, dtype=np.complex128).reshape(-1).view(np.float64)
    out[18 * N:] = np.asarray(c, dtype=np.complex128).reshape(-1).view(np.float64)
    return out


class Model:
    """Square-lattice t-t'-J model on an nx x ny torus threaded by `flux` hc/e."""

    def __init__(self, nx, ny, t=1.0, tp=-0.3, J=0.3, flux=1, gutzwiller=True, phi=None):
        self.nx, self.ny = nx, ny
        self.N = nx * ny
        self.t, self.tp, self.J = t, tp, J
        self.flux = flux
        self.gutzwiller = gutzwiller
        self.phi = peierls_phases(nx, ny, flux) if phi is None else np.asarray(phi, dtype=np.float64)
        self.fwd = neighbour_table(nx, ny, FWD)   # j = i + d
        self.nn4 = neighbour_table(nx, ny, NN4)   # j = i + e

    def hopping(self):
        """t_ij e^{i phi_ij} on the four forward bonds."""
        amp = np.array([self.t, self.t, self.tp, self.tp])[:, None]
        return amp * np.exp(1j * self.phi)


def site_factors(n, gutzwiller=True):
    """Per-site Gutzwiller factors and their derivatives.

    Returns dict with delta, m, P, gt[s], dgt[s][s'] = d g^t_s / d n_s',
    gxy, dgxy[s'] = d g^xy / d n_s'.
    """
    nu, nd = n[0], n[1]
    delta = 1.0 - nu - nd
    m = 0.5 * (nu - nd)
    P = 1.0 - delta ** 2 + 4.0 * m ** 2
    N = nu.shape[0]
    out = dict(delta=delta, m=m, P=P)
    if not gutzwiller:
        out["gt"] = np.ones((2, N))
        out["dgt"] = np.zeros((2, 2, N))
        out["gxy"] = np.ones(N)
        out["dgxy"] = np.zeros((2, N))
        return out
    clamped = delta <= CLAMP
    de = np.where(clamped, CLAMP, delta)
    Pe = 1.0 - de ** 2 + 4.0 * m ** 2
    gt = np.empty((2, N))
    dgt = np.empty((2, 2, N))
    for s, sg in ((0, 1.0), (1, -1.0)):
        up = 1.0 + de + 2.0 * sg * m
        dn = 1.0 + de - 2.0 * sg * m
        G = 2.0 * de * (1.0 - de) / Pe * up / dn
        g = np.sqrt(G)
        dlog_dd = 1.0 / de - 1.0 / (1.0 - de) + 2.0 * de / Pe + 1.0 / up - 1.0 / dn
        dlog_dd = np.where(clamped, 0.0, dlog_dd)
        dlog_dm = -8.0 * m / Pe + 2.0 * sg / up + 2.0 * sg / dn
        gt[s] = g
        for sp, sgp in ((0, 1.0), (1, -1.0)):
            dgt[s, sp] = 0.5 * g * (-dlog_dd + 0.5 * sgp * dlog_dm)
    gxy = 2.0 * (1.0 - delta) / P
    dl_dd = -1.0 / (1.0 - delta) + 2.0 * delta / P
    dl_dm = -8.0 * m / P
    dgxy = np.stack([gxy * (-dl_dd + 0.5 * dl_dm), gxy * (-dl_dd - 0.5 * dl_dm)])
    out.update(gt=gt, dgt=dgt, gxy=gxy, dgxy=dgxy)
    return out


def _ratio(A, c, X):
    """R = (A - c X^2)/(A - c) and dR/dA, dR/dc, dR/dX (reading W3)."""
    zero = c == 0.0
    Ad = np.where(A == 0.0, 1.0, A)
    den = np.where(zero, 1.0, A - c)
    R = np.where(zero, 1.0, (A - c * X ** 2) / den)
    dA = np.where(zero, 0.0, c * (X ** 2 - 1.0) / den ** 2)
    dc = np.where(zero, np.where(A == 0.0, 0.0, (1.0 - X ** 2) / Ad), A * (1.0 - X ** 2) / den ** 2)
    dX = np.where(zero, 0.0, -2.0 * c * X / den)
    return R, dA, dc, dX


def _bond_exchange(model, sf, n, chi, F, d):
    """Exchange quantities of the nn bonds i -> i + d (d = 0: +x, 1: +y)."""
    j = model.fwd[d]
    J = model.J
    gxy_ij = sf["gxy"] * sf["gxy"][j]
    cu, cd = chi[0, d], chi[1, d]
    Fij = F[d]                 # F_{i, i+d}
    Fji = F[d + 2][j]          # F_{j, j-d} = F_{j, i}
    S = abs(cu) ** 2 + abs(cd) ** 2 + abs(Fij) ** 2 + abs(Fji) ** 2
    Q = (cu * np.conj(cd) + np.conj(Fij) * Fji).real
    mi, mj = sf["m"], sf["m"][j]
    if model.gutzwiller:
        chib = 0.5 * (cu + cd)
        delb = 0.5 * (Fij + Fji)
        A = 2.0 * (abs(delb) ** 2 - abs(chib) ** 2)
        c = 4.0 * mi * mj
        Pi, Pj = sf["P"], sf["P"][j]
        di, dj = sf["delta"], sf["delta"][j]
        X = 1.0 + 12.0 * (1.0 - di) * (1.0 - dj) / np.sqrt(Pi * Pj)
        R, dRA, dRc, dRX = _ratio(A, c, X)
    else:
        N = model.N
        chib = delb = np.zeros(N, dtype=np.complex128)
        A = c = X = np.zeros(N)
        R, dRA, dRc, dRX = np.ones(N), np.zeros(N), np.zeros(N), np.zeros(N)
        di = dj = Pi = Pj = np.zeros(N)
    gz = gxy_ij * R
    Ez = J * (mi * mj - 0.25 * S)
    W = J * (gz * (mi * mj - 0.25 * S) - gxy_ij * Q)
    return dict(j=j, gxy_ij=gxy_ij, gz=gz, R=R, dRA=dRA, dRc=dRc, dRX=dRX, X=X, Ez=Ez, Q=Q,
                cu=cu, cd=cd, Fij=Fij, Fji=Fji, chib=chib, delb=delb, W=W,
                mi=mi, mj=mj, di=di, dj=dj, Pi=Pi, Pj=Pj)


def energy_W(model, params, mu, n_target=None):
    """Variational energy W (App. A) for order parameters `params`."""
    N = model.N
    n, chi, F = split(params, N)
    sf = site_factors(n, model.gutzwiller)
    tij = model.hopping()
    W = 0.0
    for d in range(4):
        j = model.fwd[d]
        for s in range(2):
            gts = sf["gt"][s] * sf["gt"][s][j]
            W -= np.sum(gts * 2.0 * (tij[d] * chi[s, d]).real)
    for d in range(2):
        W += np.sum(_bond_exchange(model, sf, n, chi, F, d)["W"])
    ntot = np.sum(n)
    Ne = N * n_target if n_target is not None else 0.0
    W -= mu * (ntot - Ne)
    return float(W)


def fields(model, params, mu):
    """Effective fields (eps, T, D) = (dW/dn, dW/dchi, dW/dF*) in the flat layout."""
    N = model.N
    n, chi, F = split(params, N)
    sf = site_factors(n, model.gutzwiller)
    tij = model.hopping()
    J = model.J
    eps = np.full((2, N), -float(mu))
    T = np.zeros((2, 4, N), dtype=np.complex128)
    D = np.zeros((4, N), dtype=np.complex128)
    sg = (1.0, -1.0)

    # hopping part, all four forward bonds
    for d in range(4):
        j = model.fwd[d]
        for s in range(2):
            T[s, d] += -sf["gt"][s] * sf["gt"][s][j] * tij[d]
            e2 = 2.0 * (tij[d] * chi[s, d]).real
            for sp in range(2):
                # d/dn_{i sp} through g^t_{i s}, and d/dn_{j sp} through g^t_{j s}
                eps[sp] += -sf["dgt"][s, sp] * sf["gt"][s][j] * e2
                np.add.at(eps[sp], j, -sf["dgt"][s, sp][j] * sf["gt"][s] * e2)

    # exchange part, nn bonds
    for d in range(2):
        b = _bond_exchange(model, sf, n, chi, F, d)
        j = b["j"]
        gz, gxy_ij = b["gz"], b["gxy_ij"]
        coefA = b["Ez"] * gxy_ij * b["dRA"]
        # dW/dchi_s
        T[0, d] += J * (-0.25 * gz * np.conj(b["cu"]) - 0.5 * gxy_ij * np.conj(b["cd"])) - coefA * np.conj(b["chib"])
        T[1, d] += J * (-0.25 * gz * np.conj(b["cd"]) - 0.5 * gxy_ij * np.conj(b["cu"])) - coefA * np.conj(b["chib"])
        # dW/dF*_ij (stored at i, e = d) and dW/dF*_ji (stored at j, e = d + 2)
        D[d] += J * (-0.25 * gz * b["Fij"] - 0.5 * gxy_ij * b["Fji"]) + coefA * b["delb"]
        np.add.at(D[d + 2], j, J * (-0.25 * gz * b["Fji"] - 0.5 * gxy_ij * b["Fij"]) + coefA * b["delb"])
        # dW/dn through m_i m_j, g^xy and R
        dWdgxy = b["Ez"] * b["R"] - J * b["Q"]
        dWdR = b["Ez"] * gxy_ij
        if model.gutzwiller:
            Xm1 = b["X"] - 1.0
            dX_ddi = Xm1 * (-1.0 / (1.0 - b["di"]) + b["di"] / b["Pi"])
            dX_ddj = Xm1 * (-1.0 / (1.0 - b["dj"]) + b["dj"] / b["Pj"])
            dX_dmi = Xm1 * (-4.0 * b["mi"] / b["Pi"])
            dX_dmj = Xm1 * (-4.0 * b["mj"] / b["Pj"])
        else:
            dX_ddi = dX_ddj = dX_dmi = dX_dmj = np.zeros(N)
        for sp in range(2):
            h = 0.5 * sg[sp]    # dm/dn_sp; d delta/dn_sp = -1
            # site i
            gi = (J * gz * b["mj"] * h
                  + dWdgxy * sf["gxy"][j] * sf["dgxy"][sp]
                  + dWdR * (b["dRc"] * 4.0 * b["mj"] * h + b["dRX"] * (-dX_ddi + h * dX_dmi)))
            eps[sp] += gi
            # site j
            gj = (J * gz * b["mi"] * h
                  + dWdgxy * sf["gxy"] * sf["dgxy"][sp][j]
                  + dWdR * (b["dRc"] * 4.0 * b["mi"] * h + b["dRX"] * (-dX_ddj + h * dX_dmj)))
            np.add.at(eps[sp], j, gj)
    return join(eps, T, D)


def mix(params, new, alpha):
    """Linear mixing p <- (1 - alpha) p + alpha p_new (reading R1)."""
    return (1.0 - alpha) * params + alpha * new


def residual(params, new):
    """Largest change of any real or imaginary parameter component (reading R1)."""
    return float(np.max(np.abs(new - params))) if params.size else 0.0


def mean_density(params, N):
    n, _, _ = split(params, N)
    return float(np.sum(n) / N)


# ----------------------------------------------------------------------------- self-consistency

def shifted_fields(model, params, mu_eff):
    """Fields with the chemical potential measured from the mean site energy.

    eps_{i s} = dW/dn_{i s}|_{mu=0} - <dW/dn|_{mu=0}> - mu_eff (reading R2): the
    Lagrange multiplier is mu = mu_eff + <dW/dn|_{mu=0}>, so the uniform part
    of the Gutzwiller site energy never enters the density feedback loop.
    Returns (fields, mu).
    """
    N = model.N
    fld = fields(model, params, 0.0)
    eps, _, _ = split(fld, N)
    eg = float(np.mean(eps))
    eps -= eg + mu_eff
    return fld, mu_eff + eg


def update(params, obs, n_target, mu_eff, alpha=0.5, alpha_n=0.05, eta=0.5, paramagnetic=True):
    """One mixing step of the RMFT loop (readings R1, R2).

      1. paramagnetic sector: n_up = n_dn = (n_up + n_dn)/2 when requested;
      2. e = <n_new> - n_target; densities shifted by -e/2 per spin;
      3. residual r = max |p_new - p| over every real and imaginary component;
      4. p <- (1 - alpha) p + alpha p_new for chi and F, with alpha_n for n;
      5. mu_eff <- mu_eff - eta e.
    Returns (params, mu_eff, r, e).
    """
    N = params.size // 26
    o = np.array(obs, dtype=np.float64, copy=True)
    if paramagnetic:
        avg = 0.5 * (o[:N] + o[N:2 * N])
        o[:N] = avg
        o[N:2 * N] = avg
    e = float(np.sum(o[:2 * N]) / N) - n_target
    o[:2 * N] -= 0.5 * e
    r = residual(params, o)
    new = (1.0 - alpha) * params + alpha * o
    new[:2 * N] = (1.0 - alpha_n) * params[:2 * N] + alpha_n * o[:2 * N]
    return new, mu_eff - eta * e, r, e


# ----------------------------------------------------------------------------- Anderson mixing (reading R4)

class Anderson:
    """Anderson (Pulay) acceleration of the fixed-point iteration x = G(x).

    The paper does not say how its self-consistency loop is mixed (reading
    R1 gives linear mixing).  Reading R4 adds the textbook Anderson scheme
    (Anderson 1965; Walker and Ni 2011), preconditioned by the linear mixing
    B (alpha_n on the densities, alpha on chi and F, eta on mu_eff):

      f_k   = B (G(x_k) - x_k)
      dX_j  = x_{j+1} - x_j,  dF_j = f_{j+1} - f_j   over the last m iterations
      gamma = argmin_g |f_k - dF g|_2   (normal equations, Tikhonov 1e-10 tr/m_k)
      x_{k+1} = x_k + f_k - (dX + dF) gamma

    With m = 0 (or no history yet) this is the linear mixing step x + f.
    """

    def __init__(self, m):
        self.m = int(m)
        self.dX, self.dF = [], []
        self.prev = None

    def step(self, x, f):
        x = np.asarray(x, dtype=np.float64)
        f = np.asarray(f, dtype=np.float64)
        if self.m > 0 and self.prev is not None:
            self.dX.append(x - self.prev[0])
            self.dF.append(f - self.prev[1])
            if len(self.dX) > self.m:
                self.dX.pop(0)
                self.dF.pop(0)
        self.prev = (x.copy(), f.copy())
        if self.m == 0 or not self.dX:
            return x + f
        dF = np.array(self.dF).T
        dX = np.array(self.dX).T
        G = dF.T @ dF
        tr = float(np.trace(G))
        if not (0.0 < tr < 1e300):
            return x + f
        G = G + 1e-10 * tr / G.shape[0] * np.eye(G.shape[0])
        gamma = np.linalg.solve(G, dF.T @ f)
        return x + f - (dX + dF) @ gamma


def update_anderson(params, obs, n_target, mu_eff, mixer, alpha=0.5, alpha_n=0.05, eta=0.5, paramagnetic=True):
    """`update` with Anderson mixing (reading R4) on x = (params, mu_eff):
    the processed observables (steps 1-2 of `update`) give G(x); the residual r
    is the same max |p_new - p| as in `update`.  Returns (params, mu_eff, r, e)."""
    N = params.size // 26
    o = np.array(obs, dtype=np.float64, copy=True)
    if paramagnetic:
        avg = 0.5 * (o[:N] + o[N:2 * N])
        o[:N] = avg
        o[N:2 * N] = avg
    e = float(np.sum(o[:2 * N]) / N) - n_target
    o[:2 * N] -= 0.5 * e
    r = residual(params, o)
    B = np.full(params.size, alpha)
    B[:2 * N] = alpha_n
    x = np.concatenate([params, [mu_eff]])
    f = np.concatenate([B * (o - params), [-eta * e]])
    xn = mixer.step(x, f)
    return xn[:-1], float(xn[-1]), r, e
