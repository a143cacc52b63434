"""Maxwell equal-area construction for the model's bulk pressure (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The coexistence densities rho_V < rho_L share one pressure p0,
p(rho_V) = p(rho_L) = p0, and satisfy the equal-area rule in specific volume
v = 1/rho: integral_{rho_V}^{rho_L} (p(rho) - p0) / rho^2 d rho = 0.  The paper
quotes the values this gives for the exponential pseudopotential (Sec. IV A)
and for the Carnahan-Starling EOS at T = 0.6 T_c (Sec. IV D, Table II).
"""

from __future__ import annotations

import numpy as np
from scipy import integrate, optimize

from .lbm_oracle import Params, eos_pressure


def _spinodals(pfun, lo, hi, n=20001):
    """The local maximum and minimum of p(rho) on (lo, hi)."""
    rho = np.linspace(lo, hi, n)
    pr = pfun(rho)
    dp = np.diff(pr)
    sign = np.sign(dp)
    idx = np.nonzero(sign[1:] != sign[:-1])[0]
    if len(idx) < 2:
        raise ValueError("no van der Waals loop: temperature above critical?")
    ext = []
    for i in idx[:2]:
        def dpdr(r):
            h = 1e-7 * max(1.0, r)
            return (pfun(r + h) - pfun(r - h)) / (2 * h)
        ext.append(optimize.brentq(dpdr, rho[i], rho[i + 2], xtol=1e-15))
    return ext[0], ext[1]


def coexistence(pfun, lo: float, hi: float):
    """(rho_L, rho_V) for a pressure function with one van der Waals loop."""
    r_max, r_min = _spinodals(pfun, lo, hi)  # p has a max at r_max < r_min
    p_hi = float(pfun(r_max))
    p_lo = max(float(pfun(r_min)), float(pfun(lo)) + 1e-300)

    def roots(p0):
        rv = optimize.brentq(lambda r: pfun(r) - p0, lo, r_max, xtol=1e-16, rtol=1e-15)
        rl = optimize.brentq(lambda r: pfun(r) - p0, r_min, hi, xtol=1e-16, rtol=1e-15)
        return rv, rl

    def area(p0):
        rv, rl = roots(p0)
        val, _ = integrate.quad(lambda r: (pfun(r) - p0) / (r * r), rv, rl,
                                epsabs=1e-14, epsrel=1e-12, limit=400)
        return val

    eps = 1e-12 * (p_hi - p_lo)
    p0 = optimize.brentq(area, p_lo + eps, p_hi - eps, xtol=1e-17, rtol=1e-15)
    rv, rl = roots(p0)
    return rl, rv


def coexistence_cs(T_over_Tc: float, a: float = 1.0, b: float = 4.0, R: float = 1.0):
    """Carnahan-Starling coexistence (rho_L, rho_V) at reduced temperature T/T_c."""
    from .lbm_oracle import critical_temperature

    p = Params(eos="cs", a=a, b=b, R=R, T=T_over_Tc * critical_temperature(a, b, R))
    return coexistence(lambda r: eos_pressure(r, p), 1e-9, 0.999 * 4.0 / b)


def coexistence_exp(G: float = -10.0 / 3.0, psi0: float = 1.0, rho0: float = 1.0):
    """Coexistence for psi = psi0 exp(-rho0/rho), p = rho/3 + G psi^2 / 2."""
    p = Params(eos="exp", G=G, psi0=psi0, rho0=rho0)
    return coexistence(lambda r: eos_pressure(r, p), 0.02, 20.0)
