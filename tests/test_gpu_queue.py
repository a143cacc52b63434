"""The single pass on the ordered work queue (lbm_set_tuning mode 5).

Fused items and the next step's psi items run in one persistent launch; their
arithmetic is that of the two-pass kernels, so every result must equal the
two-pass step bit for bit, for both operators, FP32 and FP16 storage, with
and without the Eq. 16 term, both EOS arithmetics and the exponential
pseudopotential, on cubic, non-cubic, small and odd-Ny boxes.  Also against
the FP64 oracle, and the bounded waits: an injected unreachable wait target
must come back as LBM_ERR_TIMEOUT with the context still usable.
"""

import numpy as np
import pytest

from gpu_helpers import coexistence, droplet_rho, lattice, max_abs, oracle_params, physics
from oracle import lbm_oracle as L
from relaxation_pin import SIX_RATES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_08643_gb300 import _build

    _build.build()


def _run(grid, op, prec, mode, steps, sigma=0.0, eos_arith="f64", rates=None, T=0.8, R=None):
    phys = physics(T_over_Tc=T, sigma=sigma, rates=rates)
    lat = lattice(grid, op, prec, phys)
    lat.set_tuning(mode, 1, 0)  # False: the two-pass step, explicitly (FP32 storage defaults to the work list)
    if eos_arith != "f64":
        lat.set_eos_arith(eos_arith)
    rl, rv = coexistence(T)
    lat.init_droplet(tuple(n / 2 for n in grid), R or min(grid) / 4, 2.0, rl, rv)
    lat.step(steps)
    status = lat.check()
    out = lat.moments(), lat.populations()
    lat.close()
    return status, out


def _equal(a, b):
    (ra, ua), fa = a
    (rb, ub), fb = b
    return np.array_equal(ra, rb) and np.array_equal(ua, ub) and np.array_equal(fa, fb)


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("op", ["nonorth", "orth"])
@pytest.mark.parametrize("grid", [(32, 32, 32), (24, 20, 28), (64, 18, 40), (6, 5, 7), (4, 3, 3)])
def test_queue_equals_two_pass_bit_for_bit(grid, op, prec):
    steps = 40
    s0, ref = _run(grid, op, prec, False, steps, sigma=0.105)
    s1, got = _run(grid, op, prec, "queue", steps, sigma=0.105)
    assert s0 == 0 and s1 == 0
    assert _equal(ref, got)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_queue_without_sigma_and_with_compensated_eos(prec):
    grid = (32, 24, 20)
    for kw in (dict(sigma=0.0), dict(sigma=0.105, eos_arith="f32x2")):
        s0, ref = _run(grid, "nonorth", prec, False, 30, **kw)
        s1, got = _run(grid, "nonorth", prec, "queue", 30, **kw)
        assert s0 == 0 and s1 == 0 and _equal(ref, got), kw


def test_queue_exponential_pseudopotential():
    from oracle import maxwell

    grid = (16, 16, 16)
    phys = physics(eos="exp", G=-10.0 / 3.0, other=1.2)
    phys["s_e"] = 0.8
    rl, rv = maxwell.coexistence_exp()
    rho0 = droplet_rho(grid, (8, 8, 8), 5.0, 3.0, rl, rv)
    outs = []
    for mode in (False, "queue"):
        lat = lattice(grid, "nonorth", "f32", phys)
        lat.set_tuning(mode, 1, 0)  # False: the two-pass step, explicitly (FP32 storage defaults to the work list)
        lat.init_field(rho0, rho_ref=rv)
        lat.step(30)
        assert lat.check() == 0
        outs.append((lat.moments(), lat.populations()))
        lat.close()
    assert _equal(*outs)


@pytest.mark.parametrize("op", ["nonorth", "orth"])
def test_queue_against_fp64_oracle_with_six_rates(op):
    grid, steps = (32, 32, 32), 200
    phys = physics(rates=SIX_RATES)
    rl, rv = coexistence(0.8)
    lat = lattice(grid, op, "f32", phys)
    lat.set_tuning("queue", 1, 0)
    lat.init_droplet((16.0, 16.0, 16.0), 8.0, 2.0, rl, rv)
    lat.step(steps)
    assert lat.check() == 0
    assert lat.tuning()["single_pass"] == "queue"
    rho, u = lat.moments()
    lat.close()
    p = oracle_params(grid, op, phys)
    f0 = L.equilibrium_state(p, droplet_rho(grid, (16.0, 16.0, 16.0), 8.0, 2.0, rl, rv))
    rho_o, u_o, _, _ = L.macroscopic(p, L.run(p, f0, steps))
    assert max_abs(rho, rho_o) <= 2e-5 and max_abs(u, u_o) <= 2e-5


@pytest.mark.parametrize("mode", ["queue", "lagged"])
def test_injected_unreachable_wait_times_out_and_the_context_stays_usable(mode):
    """A wait for a count no block publishes runs out its (small) budget: the kernel returns,
    lbm_check reports LBM_ERR_TIMEOUT, and after the injection is lifted the same context steps
    correctly again."""
    from paper_1805_08643_gb300.lbm import ERR_TIMEOUT

    grid = (32, 16, 12)
    rl, rv = coexistence(0.8)
    lat = lattice(grid, "nonorth", "f32", physics())
    lat.set_tuning(mode, 1, 0)
    lat.init_droplet((16.0, 8.0, 6.0), 4.0, 2.0, rl, rv)
    lat.set_wait_budget(64, inject_unreachable=True)
    lat.step(2)
    assert lat.check() == ERR_TIMEOUT
    lat.set_wait_budget(0, inject_unreachable=False)
    lat.init_droplet((16.0, 8.0, 6.0), 4.0, 2.0, rl, rv)
    lat.step(10)
    assert lat.check() == 0
    got = lat.moments(), lat.populations()
    lat.close()
    _, ref = _run(grid, "nonorth", "f32", False, 10, R=4.0)
    assert _equal(ref, got)


def test_queue_at_256_cubed_equals_two_pass():
    """The benchmark's box and launch configuration: 20 steps of the 256^3 droplet."""
    import torch

    from paper_1805_08643_gb300 import thermo
    from paper_1805_08643_gb300.lbm import Lattice, Rates

    edge, steps = 256, 20
    Tc = thermo.critical_temperature(1.0, 4.0, 1.0)
    rl, rv = thermo.coexistence_cs(0.7, 1.0, 4.0, 1.0)
    outs = []
    for mode in (False, "queue"):
        lat = Lattice((edge,) * 3, operator="nonorth", precision="f32", T=0.7 * Tc, G=-1.0,
                      rates=Rates(s_e=1.1, s_nu=1.0, s_q=1.1, s_pi=1.1, s_eps=1.1, s_m=1.1), sigma=0.105)
        lat.set_tuning(mode, 1, 0)  # False: the two-pass step, explicitly (FP32 storage defaults to the work list)
        lat.init_droplet((edge / 2,) * 3, 40.0, 3.0, rl, rv)
        lat.step(steps)
        assert lat.check() == 0
        outs.append(lat.moments())
        lat.close()
        torch.cuda.empty_cache()
    (r0, u0), (r1, u1) = outs
    assert np.array_equal(r0, r1) and np.array_equal(u0, u1)


def test_default_step_per_form():
    """FP32 storage with an even Nx steps on the work list by default (D3Q19 and D3Q15); FP16 storage, FP64
    and an odd Nx keep the two-pass step."""
    cases = [((16, 16, 16), "nonorth", "f32", "queue"), ((16, 16, 16), "orth", "f32", "queue"),
             ((16, 16, 16), "nonorth", "f16", False), ((16, 16, 16), "nonorth", "f64", False),
             ((15, 16, 16), "nonorth", "f32", False), ((16, 16, 16), "nonorth_d3q15", "f32", "queue"),
             ((16, 16, 16), "nonorth_d3q15", "f16", False)]
    for grid, op, prec, want in cases:
        lat = lattice(grid, op, prec, physics())
        assert lat.tuning()["single_pass"] == want, (grid, op, prec)
        lat.close()


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("grid", [(32, 32, 32), (24, 20, 28), (6, 5, 7)])
def test_d3q15_work_list_equals_two_pass_bit_for_bit(grid, prec):
    """The D3Q15 variant on the work list (its own fused and psi tile jobs) against its two-pass kernels."""
    steps = 30
    s0, ref = _run(grid, "nonorth_d3q15", prec, False, steps, sigma=0.105)
    s1, got = _run(grid, "nonorth_d3q15", prec, "queue", steps, sigma=0.105)
    assert s0 == 0 and s1 == 0
    assert _equal(ref, got)


def test_d3q15_work_list_against_its_oracle():
    from oracle import d3q15 as D

    grid, steps = (24, 20, 28), 200
    phys = physics(rates=SIX_RATES)
    rl, rv = coexistence(0.8)
    centre = tuple(n / 2 for n in grid)
    lat = lattice(grid, "nonorth_d3q15", "f32", phys)
    lat.set_tuning("queue", 1, 0)
    lat.init_droplet(centre, 6.0, 2.0, rl, rv)
    lat.step(steps)
    assert lat.check() == 0
    rho, u = lat.moments()
    lat.close()
    p = oracle_params(grid, "nonorth", phys)
    f0 = D.equilibrium_state(p, droplet_rho(grid, centre, 6.0, 2.0, rl, rv))
    rho_o, u_o, _, _ = D.macroscopic(p, D.run(p, f0, steps))
    assert max_abs(rho, rho_o) <= 2e-5 and max_abs(u, u_o) <= 2e-5


def test_queue_claims_stay_in_step_across_mode_switches_and_inits():
    """Blocks claim work-list items from a counter that advances with every launch: switching to the two-pass
    step and back, re-initialising, and steps in chunks of 1, 2 and 5 must leave every launch claiming its own
    items (bit-exact with the two-pass step, no LBM_ERR_TIMEOUT)."""
    grid = (32, 16, 12)
    rl, rv = coexistence(0.8)
    lat = lattice(grid, "nonorth", "f32", physics(sigma=0.105))
    lat.set_tuning("queue", 1, 0)
    lat.init_droplet((16.0, 8.0, 6.0), 4.0, 2.0, rl, rv)
    for n in (1, 2, 5):
        lat.step(n)
    lat.set_tuning(False, 1, 0)
    lat.step(3)
    lat.set_tuning("queue", 1, 0)
    lat.step(4)
    assert lat.check() == 0
    got = lat.moments(), lat.populations()
    lat.init_droplet((16.0, 8.0, 6.0), 4.0, 2.0, rl, rv)  # a new run on the same counters
    lat.step(15)
    assert lat.check() == 0
    again = lat.moments(), lat.populations()
    lat.close()
    _, ref = _run(grid, "nonorth", "f32", False, 15, sigma=0.105, R=4.0)
    assert _equal(ref, got)
    assert _equal(ref, again)
