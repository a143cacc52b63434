"""Pins for the equation of state, pseudopotentials and Maxwell construction."""

import numpy as np
import pytest

from conftest import read_values
from oracle import lbm_oracle as L
from oracle import maxwell

PAPER = read_values("paper_values.txt")


def test_maxwell_exponential_matches_paper():
    rl, rv = maxwell.coexistence_exp()
    assert abs(rl - PAPER["exp_rho_l"]) < 5e-4
    assert abs(rv - PAPER["exp_rho_v"]) < 5e-5


@pytest.mark.parametrize("a", [1.0, 0.25])
def test_maxwell_carnahan_starling_matches_paper(a):
    rl, rv = maxwell.coexistence_cs(0.6, a=a)
    assert abs(rl - PAPER["cs06_rho_l"]) < 5e-4
    assert abs(rv - PAPER["cs06_rho_v"]) < 5e-6


def test_coexistence_narrows_towards_critical_point():
    pairs = [maxwell.coexistence_cs(t) for t in (0.6, 0.7, 0.8, 0.9, 0.95)]
    gaps = [rl - rv for rl, rv in pairs]
    assert all(g1 > g2 > 0 for g1, g2 in zip(gaps, gaps[1:]))


def test_carnahan_starling_critical_point():
    # T_c = 0.37733 a/(bR) (Sec. IV D): at T_c the isotherm has a horizontal
    # inflection, dp/drho = d2p/drho2 = 0, up to the 4-digit coefficients
    # (0.4963, 0.18727) behind the constant: a slope of order 1e-4 R T.
    a, b, R = 1.0, 4.0, 1.0
    p = L.Params(eos="cs", a=a, b=b, R=R, T=L.critical_temperature(a, b, R))
    rho = np.linspace(0.05, 0.3, 250001)
    h = rho[1] - rho[0]
    pr = L.pressure_cs(rho, p)
    d1 = np.gradient(pr, h)
    d2 = np.gradient(d1, h)
    i = np.argmin(d1)
    assert abs(d1[i]) < 3e-4 * R * p.T
    assert abs(d2[i]) < 1e-2
    assert 0.12 < rho[i] < 0.14  # critical density 0.5218/b
    above = L.pressure_cs(rho, p.with_(T=1.05 * p.T))
    assert np.all(np.diff(above) > 0)  # no loop above T_c
    below = L.pressure_cs(rho, p.with_(T=0.9 * p.T))
    assert np.any(np.diff(below) < 0)


def test_carnahan_starling_ideal_gas_limit():
    p = L.Params(eos="cs", a=1.0, b=4.0, R=1.0, T=0.07)
    rho = np.array([1e-6, 1e-5])
    assert np.allclose(L.pressure_cs(rho, p), rho * p.R * p.T, rtol=1e-4)


def test_sqrt_pseudopotential_reproduces_eos_pressure():
    p = L.Params(eos="cs", T=0.7 * L.critical_temperature(1, 4, 1), G=-1.0)
    rho = np.linspace(0.005, 0.45, 50)
    psi = L.pseudopotential(rho, p)
    assert np.all(psi > 0)
    assert np.max(np.abs(rho / 3 + p.G * psi * psi / 2 - L.pressure_cs(rho, p))) < 1e-15


def test_exponential_pseudopotential():
    p = L.Params(eos="exp", psi0=1.0, rho0=1.0, G=-10 / 3)
    rho = np.array([0.5, 1.0, 2.0])
    assert np.allclose(L.pseudopotential(rho, p), np.exp(-1 / rho), rtol=0, atol=1e-16)


def test_eos_domain_errors():
    p = L.Params(eos="cs", T=0.07, G=-1.0)
    with pytest.raises(L.EOSDomainError):
        L.pseudopotential(np.array([0.1, 1.0]), p)  # b rho / 4 = 1
    with pytest.raises(L.EOSDomainError):
        L.pseudopotential(np.array([0.1, -0.1]), p)
    with pytest.raises(L.EOSDomainError):
        L.pseudopotential(np.array([0.1]), p.with_(G=1.0))  # radicand < 0
