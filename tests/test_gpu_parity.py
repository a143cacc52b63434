"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Gate: FP64, max |rho_gpu - rho_oracle| and max |u_gpu - u_oracle| <= 1e-11 after
200 steps of the 32^3 droplet workload and of a non-cubic 24x20x28 box, for both
operators.
"""

import numpy as np
import pytest

from gpu_helpers import coexistence, droplet_rho, lattice, max_abs, oracle_params, physics
from oracle import lbm_oracle as L

pytestmark = pytest.mark.gpu

OPS = ["nonorth", "orth"]
TOL_F64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_08643_gb300 import _build

    _build.build()


def _droplet_case(grid, op, precision="f64", T_over_Tc=0.8, R=8.0, W=2.0, **phys_kw):
    phys = physics(T_over_Tc=T_over_Tc, **phys_kw)
    rl, rv = coexistence(T_over_Tc)
    centre = tuple(n / 2 for n in grid)
    lat = lattice(grid, op, precision, phys)
    lat.init_droplet(centre, R, W, rl, rv)
    p = oracle_params(grid, op, phys)
    f0 = L.equilibrium_state(p, droplet_rho(grid, centre, R, W, rl, rv))
    return lat, p, f0


@pytest.mark.parametrize("op", OPS)
def test_initial_state_matches_oracle(op):
    lat, p, f0 = _droplet_case((32, 32, 32), op)
    rho, u = lat.moments()
    rho_o, u_o, _, _ = L.macroscopic(p, f0)
    assert max_abs(rho, rho_o) < 1e-14
    assert max_abs(u, u_o) < 1e-14
    assert max_abs(lat.populations(), f0) < 1e-15
    lat.close()


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("grid", [(32, 32, 32), (24, 20, 28)])
def test_fp64_parity_after_200_steps(op, grid):
    lat, p, f0 = _droplet_case(grid, op)
    lat.step(200)
    assert lat.check() == 0
    rho, u = lat.moments()
    rho_o, u_o, _, _ = L.macroscopic(p, L.run(p, f0, 200))
    err_rho, err_u = max_abs(rho, rho_o), max_abs(u, u_o)
    print(f"{op} {grid}: max|drho|={err_rho:.3e} max|du|={err_u:.3e}")
    assert err_rho <= TOL_F64 and err_u <= TOL_F64
    lat.close()


@pytest.mark.parametrize("op", OPS)
def test_single_step_each_stage(op):
    """One step from a random non-equilibrium state: all 19 populations agree."""
    grid = (8, 6, 5)
    phys = physics()
    p = oracle_params(grid, op, phys)
    rng = np.random.default_rng(7)
    rho = rng.uniform(0.05, 0.28, grid[::-1])
    u = rng.uniform(-0.02, 0.02, (3,) + grid[::-1])
    f = L.equilibrium_state(p, rho, u) + rng.normal(0, 2e-4, (19,) + grid[::-1])
    lat = lattice(grid, op, "f64", phys)
    lat.init_field(rho, rho_ref=0.02)
    lat.set_populations(f)
    assert max_abs(lat.populations(), f) < 1e-16
    lat.step(1)
    assert max_abs(lat.populations(), L.step(p, f)) < 1e-15
    lat.close()


@pytest.mark.parametrize("op", OPS)
def test_sigma_term_parity(op):
    lat, p, f0 = _droplet_case((16, 16, 16), op, R=5.0, sigma=0.105, other=1.2, s_nu=1.0 / 0.8)
    lat.step(50)
    rho, u = lat.moments()
    rho_o, u_o, _, _ = L.macroscopic(p, L.run(p, f0, 50))
    assert max_abs(rho, rho_o) <= TOL_F64 and max_abs(u, u_o) <= TOL_F64
    lat.close()


def test_exponential_pseudopotential_parity():
    grid = (16, 16, 16)
    phys = physics(eos="exp", G=-10.0 / 3.0, other=1.2)
    phys["s_e"] = 0.8
    p = oracle_params(grid, "nonorth", phys).with_(psi0=1.0, rho0=1.0)
    from oracle import maxwell

    rl, rv = maxwell.coexistence_exp()
    rho0 = droplet_rho(grid, (8, 8, 8), 5.0, 3.0, rl, rv)
    lat = lattice(grid, "nonorth", "f64", phys)
    lat.init_field(rho0, rho_ref=rv)
    lat.step(50)
    rho, u = lat.moments()
    rho_o, u_o, _, _ = L.macroscopic(p, L.run(p, L.equilibrium_state(p, rho0), 50))
    assert max_abs(rho, rho_o) <= TOL_F64 and max_abs(u, u_o) <= TOL_F64
    lat.close()


@pytest.mark.parametrize("op", OPS)
def test_flat_interface_and_mass_conservation(op):
    grid = (8, 8, 64)
    phys = physics(T_over_Tc=0.7, sigma=0.116)  # Eq. 16 keeps the 0.7 T_c slab stable
    rl, rv = coexistence(0.7)
    lat = lattice(grid, op, "f64", phys)
    lat.init_flat(2, 16.0, 48.0, 2.0, rl, rv)
    p = oracle_params(grid, op, phys)
    f0 = L.equilibrium_state(p, L.slab_density(grid, 2, 16.0, 48.0, 2.0, rl, rv))
    d0 = lat.diag()
    lat.step(100)
    d1 = lat.diag()
    rho, u = lat.moments()
    rho_o, u_o, _, _ = L.macroscopic(p, L.run(p, f0, 100))
    assert max_abs(rho, rho_o) <= TOL_F64 and max_abs(u, u_o) <= TOL_F64
    assert abs(d1["mass"] - d0["mass"]) < 1e-13 * d0["mass"]
    assert abs(d0["mass"] - L.total_mass(f0)) < 1e-12 * d0["mass"]
    assert max(abs(m) for m in d1["momentum"]) < 1e-13 * d0["mass"]
    lat.close()


def test_eos_domain_error_is_reported_not_clamped():
    grid = (8, 8, 8)
    lat = lattice(grid, "nonorth", "f64", physics())
    rho = np.full(grid[::-1], 0.2)
    rho[3, 3, 3] = 1.2  # b rho / 4 >= 1: outside the Carnahan-Starling domain
    lat.init_field(rho, rho_ref=0.2)
    lat.step(1)
    from paper_1805_08643_gb300.lbm import ERR_EOS_DOMAIN, OK

    assert lat.check() == ERR_EOS_DOMAIN
    assert lat.check() == OK  # the word is cleared by the read
    lat.close()


def test_check_interval_stops_the_step_loop():
    from paper_1805_08643_gb300.lbm import LBMError

    grid = (8, 8, 8)
    lat = lattice(grid, "orth", "f64", physics())
    rho = np.full(grid[::-1], 0.2)
    rho[1, 2, 3] = -0.1
    lat.init_field(rho, rho_ref=0.2)
    lat.set_check_interval(1)
    with pytest.raises(LBMError, match="EOS_DOMAIN"):
        lat.step(5)
    assert lat.steps == 1
    lat.close()


@pytest.mark.parametrize("op", OPS)
def test_variable_viscosity_parity(op):
    rl, rv = coexistence(0.8)
    lat, p, f0 = _droplet_case((24, 20, 28), op)
    lat.set_variable_viscosity(rl, rv, 0.05, 0.25)
    p = p.with_(nu_l=0.05, nu_v=0.25, rho_l_nu=rl, rho_v_nu=rv)
    lat.step(100)
    rho, u = lat.moments()
    rho_o, u_o, _, _ = L.macroscopic(p, L.run(p, f0, 100))
    assert max_abs(rho, rho_o) <= TOL_F64 and max_abs(u, u_o) <= TOL_F64
    lat.close()
