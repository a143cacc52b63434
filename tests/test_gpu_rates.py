"""Every relaxation rate reaches its own moments on the GPU (Eq. 4, Eq. 11, the orthogonal reading).

Two kinds of check, all through the C ABI:

* closed form: one non-conserved moment perturbed on a uniform rest state with
  G = 0 decays by (1 - s_k) in one step, with six distinct rates, for every
  row of both D3Q19 operators and of the D3Q15 variant, in the FP64 kernels
  and in the FP32 two-node kernels;
* parity with the FP64 oracle after 200 steps of a droplet with six distinct
  rates (FP64 <= 1e-11 on 32^3 and 24x20x28, FP32 two-node kernels <= 2e-5,
  one box of a batch, D3Q15).
"""

import numpy as np
import pytest

from gpu_helpers import coexistence, droplet_rho, lattice, max_abs, oracle_params, physics
from oracle import d3q15 as D
from oracle import lbm_oracle as L
from relaxation_pin import SIX_RATES, decay_error, non_conserved_rows, perturbed_rest_state

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-11
TOL_F32 = 2e-5
EPS, RHO0 = 1e-3, 0.7
# golden table name, C-ABI operator, velocities, rest weights
LATTICES = {
    "nonorth": ("nonorth", L.E, L.W_LATTICE),
    "orth": ("orth", L.E, L.W_LATTICE),
    "nonorth15": ("nonorth_d3q15", D.E, D.W_LATTICE),
}
# closed-form tolerance: FP64 rounding of the moment sums; FP32 storage rounds
# each population to ~4e-8, which the moment rows (coefficients up to 30) sum
# to a few 1e-7 -- well below the 5e-5 that separates the closest two rates
DECAY_TOL = {"f64": 1e-13, "f32": 5e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_08643_gb300 import _build

    _build.build()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("op_name", ["nonorth", "orth", "nonorth15"])
def test_each_moment_decays_with_its_own_rate(op_name, prec):
    from paper_1805_08643_gb300.lbm import Lattice, Rates

    op, E, w = LATTICES[op_name]
    grid = (4, 4, 4)  # even Nx: the FP32 form runs the two-node kernels
    lat = Lattice(grid, operator=op, precision=prec, eos="none", G=0.0, rates=Rates(**SIX_RATES))
    lat.init_field(np.full(grid[::-1], RHO0), rho_ref=RHO0)
    worst = {}
    for k in non_conserved_rows(op_name):
        f0 = perturbed_rest_state(op_name, E, w, k, EPS, RHO0, grid)
        lat.set_populations(f0)
        f0_stored = lat.populations()  # rounded to the storage precision
        lat.step(1)
        worst[k] = decay_error(op_name, E, f0_stored, lat.populations(), k, EPS, SIX_RATES, 1)
    assert lat.check() == 0
    lat.close()
    bad = {k: v for k, v in worst.items() if v > DECAY_TOL[prec]}
    assert not bad, f"{op_name} {prec}: rows decaying with the wrong rate: {bad}"


def _droplet(grid, op, prec, R=8.0, W=2.0, oracle=L):
    phys = physics(rates=SIX_RATES)
    rl, rv = coexistence(0.8)
    centre = tuple(n / 2 for n in grid)
    lat = lattice(grid, op, prec, phys)
    lat.init_droplet(centre, R, W, rl, rv)
    oop = "nonorth" if op == "nonorth_d3q15" else op
    p = oracle_params(grid, oop, phys)
    f0 = oracle.equilibrium_state(p, droplet_rho(grid, centre, R, W, rl, rv))
    return lat, p, f0


@pytest.mark.parametrize("op", ["nonorth", "orth"])
@pytest.mark.parametrize("grid", [(32, 32, 32), (24, 20, 28)])
def test_fp64_parity_with_six_distinct_rates(op, grid):
    lat, p, f0 = _droplet(grid, op, "f64")
    lat.step(200)
    assert lat.check() == 0
    rho, u = lat.moments()
    lat.close()
    rho_o, u_o, _, _ = L.macroscopic(p, L.run(p, f0, 200))
    err_r, err_u = max_abs(rho, rho_o), max_abs(u, u_o)
    print(f"{op} {grid} six rates: max|drho|={err_r:.3e} max|du|={err_u:.3e}")
    assert err_r <= TOL_F64 and err_u <= TOL_F64


@pytest.mark.parametrize("op", ["nonorth", "orth"])
def test_fp32_pair_kernels_with_six_distinct_rates(op):
    grid = (32, 32, 32)
    lat, p, f0 = _droplet(grid, op, "f32")
    lat.step(200)
    assert lat.check() == 0
    rho, u = lat.moments()
    lat.close()
    rho_o, u_o, _, _ = L.macroscopic(p, L.run(p, f0, 200))
    assert max_abs(rho, rho_o) <= TOL_F32 and max_abs(u, u_o) <= TOL_F32


@pytest.mark.parametrize("op", ["nonorth", "orth"])
def test_batched_box_with_six_distinct_rates(op):
    """The batch carries each box's rates in its descriptor table: one box against the oracle."""
    from paper_1805_08643_gb300.lbm import Batch, Rates

    grid, steps = (24, 20, 28), 100
    phys = physics(rates=SIX_RATES)
    rl, rv = coexistence(0.8)
    centre = tuple(n / 2 for n in grid)
    b = Batch("f32", "cs", 1 << 34)
    # a neighbour with the default rates, so that a crossed descriptor would show
    other = b.add((32, 32, 32), "nonorth", a=phys["a"], b=phys["b"], R=phys["R"], T=phys["T"], G=phys["G"],
                  rates=Rates(), sigma=0.0)
    b.init_droplet(other, (16.0, 16.0, 16.0), 8.0, 2.0, rl, rv)
    box = b.add(grid, op, a=phys["a"], b=phys["b"], R=phys["R"], T=phys["T"], G=phys["G"],
                rates=Rates(**SIX_RATES), sigma=0.0)
    b.init_droplet(box, centre, 6.0, 2.0, rl, rv)
    b.step(steps)
    assert b.check() == 0
    rho, u = b.moments(box)
    b.close()
    p = oracle_params(grid, op, phys)
    f0 = L.equilibrium_state(p, droplet_rho(grid, centre, 6.0, 2.0, rl, rv))
    rho_o, u_o, _, _ = L.macroscopic(p, L.run(p, f0, steps))
    assert max_abs(rho, rho_o) <= TOL_F32 and max_abs(u, u_o) <= TOL_F32


@pytest.mark.parametrize("prec,tol", [("f64", TOL_F64), ("f32", TOL_F32)])
def test_d3q15_with_six_distinct_rates(prec, tol):
    grid = (24, 20, 28)
    lat, p, f0 = _droplet(grid, "nonorth_d3q15", prec, R=6.0, oracle=D)
    lat.step(200)
    assert lat.check() == 0
    rho, u = lat.moments()
    lat.close()
    rho_o, u_o, _, _ = D.macroscopic(p, D.run(p, f0, 200))
    assert max_abs(rho, rho_o) <= tol and max_abs(u, u_o) <= tol
