"""Coexistence densities used to build initial states (host-side set-up).

The initial tanh profiles of Eq. 59 and of the flat slab need the liquid and
vapour densities of the chosen equation of state.  They follow from equal
pressure and equal chemical potential of the two phases, which is the Maxwell
equal-area rule (Sec. IV A, IV D) written as two algebraic equations, solved
here by nested bisection (pressure of coexistence outside, the two
branches of the isotherm inside):

* Carnahan-Starling (Eq. 58), eta = b rho / 4:
  mu(rho) = RT ln(rho) + RT (8 eta - 9 eta^2 + 3 eta^3)/(1 - eta)^3 - 2 a rho
* exponential pseudopotential psi = psi0 exp(-rho0/rho), p = rho/3 + G psi^2/2
  (Sec. II B): the equal-area rule in 1/rho gives
  mu(rho) = ln(rho)/3 + (G psi0^2 / (2 rho0)) (rho0/rho + 1/2) exp(-2 rho0/rho),
  the integral of dp / rho.
"""

from __future__ import annotations

import math


def critical_temperature(a: float, b: float, R: float) -> float:
    """T_c = 0.37733 a / (b R) as the paper states for the C-S EOS (Sec. IV D)."""
    return 0.37733 * a / (b * R)


def _cs(a, b, RT):
    def p(r):
        e = 0.25 * b * r
        return r * RT * (1 + e + e * e - e ** 3) / (1 - e) ** 3 - a * r * r

    def mu(r):
        e = 0.25 * b * r
        return RT * math.log(r) + RT * (8 * e - 9 * e * e + 3 * e ** 3) / (1 - e) ** 3 - 2 * a * r

    return p, mu


def _exp(G, psi0, rho0):
    def p(r):
        return r / 3 + 0.5 * G * psi0 * psi0 * math.exp(-2 * rho0 / r)

    def mu(r):  # integral of dp / rho
        return math.log(r) / 3 + 0.5 * G * psi0 * psi0 * (rho0 / r + 0.5) * math.exp(-2 * rho0 / r) / rho0

    return p, mu


def _bisect(fn, lo, hi, iters=200):
    flo = fn(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = fn(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi - lo <= 1e-15 * max(1.0, abs(hi)):
            break
    return 0.5 * (lo + hi)


def _solve(p, mu, lo, hi, n=4000):
    """Equal p and equal mu: nested bisection in the pressure of coexistence."""
    # spinodals: the local maximum r_a and minimum r_b of p on a log-spaced scan
    rs = [lo * (hi / lo) ** (k / n) for k in range(n + 1)]
    ps = [p(r) for r in rs]
    turns = [k for k in range(1, n) if (ps[k] - ps[k - 1]) * (ps[k + 1] - ps[k]) < 0]
    if len(turns) < 2:
        raise ValueError("no van der Waals loop at this temperature")

    def dp(r):
        h = 1e-7 * r
        return p(r + h) - p(r - h)

    r_a = _bisect(dp, rs[turns[0] - 1], rs[turns[0] + 1])
    r_b = _bisect(dp, rs[turns[1] - 1], rs[turns[1] + 1])

    def branches(p0):
        rv = _bisect(lambda r: p(r) - p0, lo, r_a)
        rl = _bisect(lambda r: p(r) - p0, r_b, hi)
        return rv, rl

    def gap(p0):
        rv, rl = branches(p0)
        return mu(rl) - mu(rv)

    p_hi = p(r_a)
    p_lo = max(p(r_b), p(lo))
    eps = 1e-13 * (p_hi - p_lo)
    p0 = _bisect(gap, p_lo + eps, p_hi - eps)
    rv, rl = branches(p0)
    return rl, rv


def coexistence_cs(T_over_Tc: float, a: float = 1.0, b: float = 4.0, R: float = 1.0):
    """(rho_L, rho_V) of the Carnahan-Starling EOS at reduced temperature T/T_c < 1."""
    if not 0.3 < T_over_Tc < 0.995:
        raise ValueError("T/T_c must lie in (0.3, 0.995)")
    T = T_over_Tc * critical_temperature(a, b, R)
    p, mu = _cs(a, b, R * T)
    return _solve(p, mu, 1e-10, 0.999 * 4.0 / b)


def coexistence_exp(G: float = -10.0 / 3.0, psi0: float = 1.0, rho0: float = 1.0):
    """(rho_L, rho_V) of the exponential pseudopotential."""
    p, mu = _exp(G, psi0, rho0)
    return _solve(p, mu, 0.02 * rho0, 20.0 * rho0)
