"""Textbook references used to pin the oracle (independent of the paper's curvilinear forms).

* HLLC with Davis wave speeds in x: Toro, Riemann Solvers and Numerical Methods
  for Fluid Dynamics, 3rd ed., Sec. 10.4-10.6.
* Exact Riemann solver for the 1D Euler equations: Toro, Ch. 4 (pressure
  function with Newton iteration, sampling of the self-similar solution).
* Primitive-variable characteristic variables of the 1D Euler equations in x:
  dp - rho a du (u - a), a^2 drho - dp, dv, dw (u), dp + rho a du (u + a).
"""
import math

import numpy as np


def toro_hllc_x(PL, PR, gamma=1.4):
    def parts(P):
        rho, u, v, w, p = P
        E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)
        a = math.sqrt(gamma * p / rho)
        U = np.array([rho, rho * u, rho * v, rho * w, E])
        F = np.array([rho * u, rho * u * u + p, rho * u * v, rho * u * w, u * (E + p)])
        return rho, u, v, w, p, E, a, U, F

    rl, ul, vl, wl, pl, El, al, Ul, Fl = parts(PL)
    rr, ur, vr, wr, pr, Er, ar, Ur, Fr = parts(PR)
    SL = min(ul - al, ur - ar)
    SR = max(ul + al, ur + ar)
    Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) / (rl * (SL - ul) - rr * (SR - ur))

    def ustar(rho, u, v, w, p, E, S):
        f = rho * (S - u) / (S - Ss)
        return f * np.array([1.0, Ss, v, w, E / rho + (Ss - u) * (Ss + p / (rho * (S - u)))])

    if SL >= 0:
        return Fl
    if Ss >= 0:
        return Fl + SL * (ustar(rl, ul, vl, wl, pl, El, SL) - Ul)
    if SR > 0:
        return Fr + SR * (ustar(rr, ur, vr, wr, pr, Er, SR) - Ur)
    return Fr


def char_matrices_x(rho, p, gamma=1.4):
    """Left eigenvector rows (as listed in the module docstring) and their inverse."""
    a = math.sqrt(gamma * p / rho)
    Lm = np.array([[0.0, -rho * a, 0, 0, 1], [a * a, 0, 0, 0, -1], [0, 0, 1, 0, 0], [0, 0, 0, 1, 0],
                   [0.0, rho * a, 0, 0, 1]])
    return Lm, np.linalg.inv(Lm)


def exact_riemann(rl, ul, pl, rr, ur, pr, gamma, xi):
    """Exact solution (rho, u, p) of the 1D Riemann problem sampled at xi = x/t (Toro Ch. 4)."""
    al, ar = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1) / (2 * gamma)

    def fk(p, rk, pk, ak):
        if p > pk:
            A = 2 / ((gamma + 1) * rk)
            B = (gamma - 1) / (gamma + 1) * pk
            f = (p - pk) * math.sqrt(A / (p + B))
            df = math.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
        else:
            f = 2 * ak / (gamma - 1) * ((p / pk) ** g1 - 1)
            df = 1 / (rk * ak) * (p / pk) ** (-(gamma + 1) / (2 * gamma))
        return f, df

    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        f1, d1 = fk(p, rl, pl, al)
        f2, d2 = fk(p, rr, pr, ar)
        dp = (f1 + f2 + ur - ul) / (d1 + d2)
        p = max(1e-10, p - dp)
        if abs(dp) < 1e-14 * p:
            break
    f1, _ = fk(p, rl, pl, al)
    f2, _ = fk(p, rr, pr, ar)
    us = 0.5 * (ul + ur) + 0.5 * (f2 - f1)
    out = np.zeros((3, len(xi)))
    gm = (gamma - 1) / (gamma + 1)
    for n, s in enumerate(xi):
        if s <= us:  # left of contact
            if p > pl:
                rs = rl * ((p / pl + gm) / (gm * p / pl + 1))
                S = ul - al * math.sqrt((gamma + 1) / (2 * gamma) * p / pl + g1)
                out[:, n] = (rl, ul, pl) if s < S else (rs, us, p)
            else:
                rs = rl * (p / pl) ** (1 / gamma)
                ash = al * (p / pl) ** g1
                if s < ul - al:
                    out[:, n] = (rl, ul, pl)
                elif s > us - ash:
                    out[:, n] = (rs, us, p)
                else:
                    u = 2 / (gamma + 1) * (al + (gamma - 1) / 2 * ul + s)
                    c = 2 / (gamma + 1) * (al + (gamma - 1) / 2 * (ul - s))
                    out[:, n] = (rl * (c / al) ** (2 / (gamma - 1)), u, pl * (c / al) ** (1 / g1))
        else:
            if p > pr:
                rs = rr * ((p / pr + gm) / (gm * p / pr + 1))
                S = ur + ar * math.sqrt((gamma + 1) / (2 * gamma) * p / pr + g1)
                out[:, n] = (rr, ur, pr) if s > S else (rs, us, p)
            else:
                rs = rr * (p / pr) ** (1 / gamma)
                ash = ar * (p / pr) ** g1
                if s > ur + ar:
                    out[:, n] = (rr, ur, pr)
                elif s < us + ash:
                    out[:, n] = (rs, us, p)
                else:
                    u = 2 / (gamma + 1) * (-ar + (gamma - 1) / 2 * ur + s)
                    c = 2 / (gamma + 1) * (ar - (gamma - 1) / 2 * (ur - s))
                    out[:, n] = (rr * (c / ar) ** (2 / (gamma - 1)), u, pr * (c / ar) ** (1 / g1))
    return out
