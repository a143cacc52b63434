"""The paper's validation experiments, on the GPU (FP32 arithmetic).

* Table I (Sec. IV A): 120^3 phase separation, psi = exp(-1/rho), G = -10/3,
  s_e = 0.8, nu = 0.1, other rates 1.2, rho = 1 - U[0,10]/5000, t = 8000:
  rho_L ~ 2.79-2.80, rho_V ~ 0.365-0.369 for both operators.
* Table II (Sec. IV D): 120^3 droplet r0 = 40, T = 0.6 T_c, a = 0.25, W = 5,
  sigma = 0.105: rho_L = 0.408 and rho_V ~ 0.0030-0.0032; max spurious |u|
  below 0.005 for 1/s_nu >= 0.65.
* Laplace law (Sec. IV B, Fig. 2): Delta p linear in 1/R_d for several radii.
* The D3Q15 variant (Sec. II A) on the Table I and Table II set-ups: the same
  coexistence densities; its spurious currents are larger than D3Q19's.
"""

import numpy as np
import pytest

from conftest import read_values

pytestmark = pytest.mark.gpu

PAPER = read_values("paper_values.txt")


def _build():
    from paper_1805_08643_gb300 import _build as b

    b.build()


@pytest.mark.parametrize("op", ["nonorth", "orth", "nonorth_d3q15"])
def test_table1_phase_separation(op):
    _build()
    from paper_1805_08643_gb300.lbm import Lattice, Rates

    n = 120
    rng = np.random.default_rng(1805)
    rho0 = 1.0 - rng.uniform(0.0, 10.0, (n, n, n)) / 5000.0
    nu = 0.1
    rates = Rates(s_e=0.8, s_nu=1.0 / (3 * nu + 0.5), s_q=1.2, s_pi=1.2, s_eps=1.2, s_m=1.2)
    lat = Lattice((n, n, n), operator=op, precision="f32", eos="exp", psi0=1.0, rho0=1.0, G=-10.0 / 3.0,
                  rates=rates)
    lat.init_field(rho0, rho_ref=1.0)
    lat.step(8000)
    assert lat.check() == 0
    rho, u = lat.moments()
    lat.close()
    rho_l, rho_v = float(np.percentile(rho, 99.9)), float(np.percentile(rho, 0.1))
    print(f"Table I {op}: rho_L={rho_l:.4f} rho_V={rho_v:.4f} (paper ~2.79-2.80 / 0.365-0.369)")
    assert abs(rho_l - 2.797) < 0.02 and abs(rho_v - 0.367) < 0.01
    assert abs(rho_l - PAPER["exp_rho_l"]) < 0.03  # Maxwell value printed in Sec. IV A


@pytest.mark.parametrize("op", ["nonorth", "orth"])
def test_table2_droplet_coexistence_and_spurious_currents(op):
    _build()
    from paper_1805_08643_gb300 import thermo
    from paper_1805_08643_gb300.lbm import Lattice, Rates

    n, a = 120, 0.25
    Tc = thermo.critical_temperature(a, 4.0, 1.0)
    rl, rv = thermo.coexistence_cs(0.6, a, 4.0, 1.0)
    nu = 0.1
    rates = Rates(s_e=0.8, s_nu=1.0 / (3 * nu + 0.5), s_q=1.2, s_pi=1.2, s_eps=1.2, s_m=1.2)
    lat = Lattice((n, n, n), operator=op, precision="f32", eos="cs", a=a, T=0.6 * Tc, G=-1.0, rates=rates,
                  sigma=0.105)
    lat.init_droplet((n / 2,) * 3, 40.0, 5.0, rl, rv)
    lat.step(10000)
    assert lat.check() == 0
    rho, u = lat.moments()
    lat.close()
    c = n // 2
    rho_l, rho_v = float(rho[c, c, c]), float(rho[0, 0, 0])
    umax = float(np.sqrt((u * u).sum(0)).max())
    print(f"Table II {op}: rho_L={rho_l:.4f} rho_V={rho_v:.5f} max|u|={umax:.4f} "
          "(paper 0.408 / 0.0030-0.0032, < 0.005)")
    assert abs(rho_l - 0.408) < 0.004
    assert 0.0028 < rho_v < 0.0034
    assert umax < 0.005


def test_table2_droplet_coexistence_d3q15():
    """Table II on the D3Q15 variant: the densities the paper prints for D3Q19.

    Its spurious currents are about three times those of D3Q19 (the smaller
    velocity set, Sec. II A); the paper's < 0.005 applies to its D3Q19 model,
    so here they are only checked to stay of that order."""
    _build()
    from paper_1805_08643_gb300 import thermo
    from paper_1805_08643_gb300.lbm import Lattice, Rates

    n, a = 120, 0.25
    Tc = thermo.critical_temperature(a, 4.0, 1.0)
    rl, rv = thermo.coexistence_cs(0.6, a, 4.0, 1.0)
    rates = Rates(s_e=0.8, s_nu=1.0 / 0.8, s_q=1.2, s_pi=1.2, s_eps=1.2, s_m=1.2)
    lat = Lattice((n, n, n), operator="nonorth_d3q15", precision="f32", eos="cs", a=a, T=0.6 * Tc, G=-1.0,
                  rates=rates, sigma=0.105)
    lat.init_droplet((n / 2,) * 3, 40.0, 5.0, rl, rv)
    lat.step(10000)
    assert lat.check() == 0
    rho, u = lat.moments()
    lat.close()
    c = n // 2
    rho_l, rho_v = float(rho[c, c, c]), float(rho[0, 0, 0])
    umax = float(np.sqrt((u * u).sum(0)).max())
    print(f"Table II D3Q15: rho_L={rho_l:.4f} rho_V={rho_v:.5f} max|u|={umax:.4f}")
    assert abs(rho_l - 0.408) < 0.004
    assert 0.0028 < rho_v < 0.0034
    assert umax < 0.02


def test_laplace_law_both_operators_in_one_batch():
    """Delta p against 1/R_d is a line through the origin; both operators agree.

    Sec. IV B setup (exponential pseudopotential, s_e = 0.8, nu = 0.1, other
    rates 1.2) on 80^3 boxes, radii 12-24, all eight runs in one batch.
    """
    _build()
    from paper_1805_08643_gb300 import thermo
    from paper_1805_08643_gb300.lbm import Batch, Rates

    n, G = 80, -10.0 / 3.0
    rl, rv = thermo.coexistence_exp(G)
    rates = Rates(s_e=0.8, s_nu=1.25, s_q=1.2, s_pi=1.2, s_eps=1.2, s_m=1.2)
    radii = [12.0, 16.0, 20.0, 24.0]
    batch = Batch("f32", "exp", 1 << 36)
    boxes = {}
    for op in ("nonorth", "orth"):
        for R in radii:
            b = batch.add((n, n, n), op, psi0=1.0, rho0=1.0, G=G, rates=rates)
            batch.init_droplet(b, (n / 2,) * 3, R, 3.0, rl, rv)
            boxes[(op, R)] = b
    batch.step(8000)
    assert batch.check() == 0

    def p_eos(r):  # rho c_s^2 + G psi^2 / 2 with psi = exp(-1/rho)
        return r / 3.0 + 0.5 * G * np.exp(-2.0 / r)

    fits = {}
    for op in ("nonorth", "orth"):
        xs, ys = [], []
        for R in radii:
            rho, _ = batch.moments(boxes[(op, R)])
            c = n // 2
            r_in, r_out = float(rho[c, c, c]), float(rho[0, 0, 0])
            vol = float(((rho - r_out) / (r_in - r_out)).sum())
            Rd = (3 * vol / (4 * np.pi)) ** (1 / 3)
            xs.append(1.0 / Rd)
            ys.append(p_eos(r_in) - p_eos(r_out))
        k, c0 = np.polyfit(xs, ys, 1)
        pred = k * np.array(xs) + c0
        r2 = 1 - np.sum((np.array(ys) - pred) ** 2) / np.sum((np.array(ys) - np.mean(ys)) ** 2)
        fits[op] = (k, c0, r2)
        print(f"Laplace {op}: R_d={[round(1 / x, 2) for x in xs]} dp={[f'{y:.3e}' for y in ys]} "
              f"surface tension ~ {k / 2:.4e}, intercept {c0:.2e}, R^2 {r2:.5f}")
        assert r2 > 0.99
        assert abs(c0) < 0.1 * k * min(xs)
    batch.close()
    assert abs(fits["nonorth"][0] / fits["orth"][0] - 1) < 0.03


def test_viscosity_ratio_reduces_spurious_currents():
    """Sec. IV D: with nu_L = 0.01 (1/s_nu = 0.53), raising nu_V / nu_L from 1 to 10
    lowers the maximum spurious velocity from about 0.04 to about 0.006.

    Started directly at nu = 0.01 from the W = 5 tanh profile the run diverges
    within 500 steps, in FP64 as well; the paper does not say how it started.
    Here the droplet first relaxes 3000 steps at nu = 0.1, then the viscosity is
    switched (lbm_set_variable_viscosity; equal values give a constant nu).
    """
    _build()
    from paper_1805_08643_gb300 import thermo
    from paper_1805_08643_gb300.lbm import Lattice, Rates

    n, a = 120, 0.25
    Tc = thermo.critical_temperature(a, 4.0, 1.0)
    rl, rv = thermo.coexistence_cs(0.6, a, 4.0, 1.0)
    nu_l = 0.01
    umax = {}
    for ratio in (1.0, 10.0):
        rates = Rates(s_e=0.8, s_nu=1.0 / (3 * 0.1 + 0.5), s_q=1.2, s_pi=1.2, s_eps=1.2, s_m=1.2)
        lat = Lattice((n, n, n), operator="nonorth", precision="f32", eos="cs", a=a, T=0.6 * Tc, G=-1.0,
                      rates=rates, sigma=0.105)
        lat.init_droplet((n / 2,) * 3, 40.0, 5.0, rl, rv)
        lat.step(3000)
        lat.set_variable_viscosity(rl, rv, nu_l, ratio * nu_l)
        lat.step(10000)
        assert lat.check() == 0
        rho, u = lat.moments()
        lat.close()
        umax[ratio] = float(np.sqrt((u * u).sum(0)).max())
    print(f"spurious max|u| at nu_L = 0.01: nu_V/nu_L = 1: {umax[1.0]:.4f}, = 10: {umax[10.0]:.4f} "
          "(paper ~0.04 -> ~0.006)")
    assert 0.02 < umax[1.0] < 0.08
    assert umax[10.0] < 0.015 and umax[10.0] < 0.3 * umax[1.0]
