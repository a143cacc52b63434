"""Shared set-up of the GPU parity tests: the same seeded inputs for both sides."""

import numpy as np

from oracle import lbm_oracle as L
from oracle import maxwell

A, B, R_GAS = 1.0, 4.0, 1.0


def physics(T_over_Tc=0.8, s_nu=1.0, other=1.1, G=-1.0, sigma=0.0, eos="cs", rates=None):
    """Carnahan-Starling droplet physics of the 32^3 parity workload.

    rates: a dict of relaxation rates (s_e, s_nu, s_q, s_pi, s_eps, s_m) that replaces
    the s_nu / other pair, e.g. six distinct rates.
    """
    Tc = L.critical_temperature(A, B, R_GAS)
    d = dict(eos=eos, a=A, b=B, R=R_GAS, T=T_over_Tc * Tc, G=G, sigma=sigma,
             s_e=other, s_nu=s_nu, s_q=other, s_pi=other, s_eps=other, s_m=other)
    if rates:
        d.update(rates)
    return d


def oracle_params(grid, op, phys):
    return L.Params(grid=tuple(grid), operator=op, **phys)


def lattice(grid, op, precision, phys, **kw):
    from paper_1805_08643_gb300.lbm import Lattice, Rates

    rates = Rates(phys["s_e"], phys["s_nu"], phys["s_q"], phys["s_pi"], phys["s_eps"], phys["s_m"])
    return Lattice(grid, operator=op, precision=precision, eos=phys["eos"], a=phys["a"], b=phys["b"],
                   R=phys["R"], T=phys["T"], G=phys["G"], rates=rates, sigma=phys["sigma"], **kw)


def coexistence(T_over_Tc):
    return maxwell.coexistence_cs(T_over_Tc, a=A, b=B, R=R_GAS)


def droplet_rho(grid, centre, R, W, rl, rv):
    return L.droplet_density(tuple(grid), centre, R, W, rl, rv)


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))
