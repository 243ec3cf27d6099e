"""Exact reference solutions used by the pin tests (written from textbook
definitions; no DG arithmetic).

* ``sod_exact``: exact solution of the 1D Riemann problem for an ideal gas
  (the two-rarefaction/shock pressure function solved by Newton's method,
  then sampled along x/t), after Toro, "Riemann Solvers and Numerical Methods
  for Fluid Dynamics", Ch. 4.
"""
import math

import numpy as np


def _f_side(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1) * rho)
        B = (g - 1) / (g + 1) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
    else:  # rarefaction
        f = 2 * ck / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1) / (2 * g))
    return f, df


def sod_exact(x, t, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=0.0, g=1.4):
    """(rho, u, p) of the exact Riemann solution at positions x, time t > 0."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    p = 0.5 * (pL + pR)
    for _ in range(100):
        fL, dL = _f_side(p, rL, pL, cL, g)
        fR, dR = _f_side(p, rR, pR, cR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-15 * p:
            break
    fL, _ = _f_side(p, rL, pL, cL, g)
    fR, _ = _f_side(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    out = np.zeros((len(x), 3))
    for idx, xx in enumerate(x):
        s = (xx - x0) / t
        if s <= u:  # left of contact
            if p > pL:
                rs = rL * ((p / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pL + 1))
                S = uL - cL * math.sqrt((g + 1) / (2 * g) * p / pL + (g - 1) / (2 * g))
                out[idx] = (rL, uL, pL) if s < S else (rs, u, p)
            else:
                cs = cL * (p / pL) ** ((g - 1) / (2 * g))
                rs = rL * (p / pL) ** (1 / g)
                if s < uL - cL:
                    out[idx] = (rL, uL, pL)
                elif s > u - cs:
                    out[idx] = (rs, u, p)
                else:
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    uu = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    rr = rL * (c / cL) ** (2 / (g - 1))
                    out[idx] = (rr, uu, pL * (c / cL) ** (2 * g / (g - 1)))
        else:  # right of contact
            if p > pR:
                rs = rR * ((p / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pR + 1))
                S = uR + cR * math.sqrt((g + 1) / (2 * g) * p / pR + (g - 1) / (2 * g))
                out[idx] = (rR, uR, pR) if s > S else (rs, u, p)
            else:
                cs = cR * (p / pR) ** ((g - 1) / (2 * g))
                rs = rR * (p / pR) ** (1 / g)
                if s > uR + cR:
                    out[idx] = (rR, uR, pR)
                elif s < u + cs:
                    out[idx] = (rs, u, p)
                else:
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    uu = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    rr = rR * (c / cR) ** (2 / (g - 1))
                    out[idx] = (rr, uu, pR * (c / cR) ** (2 * g / (g - 1)))
    return out
