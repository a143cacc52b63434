"""The single pass in which the next psi pass trails the fused pass (set_tuning("lagged")).

* Against the FP64 oracle with the tolerances of the FP32-arithmetic forms
  (derived in test_gpu_precision.py): 2e-5 (FP32), 2e-3 (FP16 storage).
* Against the two-pass step: the same per-node arithmetic in the same order,
  so the cooperative launch, the z chunks and the order of the planes change
  nothing (bit for bit, FP32 and FP16 storage).  Boxes smaller than a tile,
  ragged tiles in x and y, thin boxes and many chunks are included.
"""

import numpy as np
import pytest

from gpu_helpers import coexistence, droplet_rho, lattice, max_abs, oracle_params, physics
from oracle import lbm_oracle as L

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-5, "f16": 2e-3}
OPS = ["nonorth", "orth"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1805_08643_gb300 import _build

    _build.build()


def _run(grid, op, prec, steps, mode, eos_arith="f64", sigma=0.0, R=8.0):
    phys = physics(T_over_Tc=0.8, sigma=sigma)
    rl, rv = coexistence(0.8)
    lat = lattice(grid, op, prec, phys)
    lat.set_tuning(mode, 1, 0)  # False: the two-pass step, explicitly (FP32 storage defaults to the work list)
    lat.set_eos_arith(eos_arith)
    lat.init_droplet(tuple(n / 2 for n in grid), R, 2.0, rl, rv)
    d0 = lat.diag()
    lat.step(steps)
    d1 = lat.diag()
    rho, u = lat.moments()
    st = lat.check()
    f = lat.populations()
    lat.close()
    return rho, u, f, d0, d1, st


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("grid", [(32, 32, 32), (24, 20, 28)])
def test_lagged_against_fp64_oracle(prec, op, grid):
    phys = physics(T_over_Tc=0.8)
    rl, rv = coexistence(0.8)
    p = oracle_params(grid, op, phys)
    c = tuple(n / 2 for n in grid)
    f = L.run(p, L.equilibrium_state(p, droplet_rho(grid, c, 8.0, 2.0, rl, rv)), 200)
    rho_o, u_o = L.macroscopic(p, f)[:2]
    rho, u, _, d0, d1, st = _run(grid, op, prec, 200, "lagged")
    assert st == 0
    err_r, err_u = max_abs(rho, rho_o), max_abs(u, u_o)
    print(f"lagged {prec} {op} {grid}: |drho|={err_r:.2e} |du|={err_u:.2e}")
    assert err_r <= TOL[prec] and err_u <= TOL[prec]
    assert abs(d1["mass"] - d0["mass"]) <= 20 * TOL[prec] * d0["mass"] / 19


@pytest.mark.parametrize("grid", [(32, 32, 32), (40, 36, 30), (72, 24, 20), (16, 16, 16), (6, 5, 4), (4, 3, 3),
                                  (64, 16, 48)])
@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("eos_arith", ["f64", "f32x2"])
def test_lagged_equals_two_pass(grid, prec, eos_arith):
    for op in OPS:
        R = min(8.0, min(grid) / 3)
        a = _run(grid, op, prec, 30, "lagged", eos_arith=eos_arith, sigma=0.1, R=R)
        b = _run(grid, op, prec, 30, False, eos_arith=eos_arith, sigma=0.1, R=R)
        assert a[5] == 0 and b[5] == 0
        assert np.array_equal(a[2], b[2]), (op, max_abs(a[2], b[2]))


def test_lagged_long_run_on_a_multi_chunk_box():
    """Many tiles and z chunks, 200 steps: still the two-pass result (FP32, bit for bit)."""
    a = _run((96, 64, 128), "nonorth", "f32", 200, "lagged", sigma=0.105, R=20.0)
    b = _run((96, 64, 128), "nonorth", "f32", 200, False, sigma=0.105, R=20.0)
    assert a[5] == 0 and b[5] == 0
    assert np.array_equal(a[2], b[2])


def test_lagged_reports_eos_domain_errors():
    from paper_1805_08643_gb300.lbm import ERR_EOS_DOMAIN, OK

    grid = (8, 8, 8)
    lat = lattice(grid, "nonorth", "f32", physics())
    lat.set_tuning("lagged")
    rho = np.full(grid[::-1], 0.2)
    rho[3, 3, 3] = 1.2  # b rho / 4 >= 1: outside the Carnahan-Starling domain
    lat.init_field(rho, rho_ref=0.2)
    lat.step(1)
    # the step also evaluates psi of the next state, from populations the NaN psi
    # has already reached: the non-finite bit is set too and takes precedence
    from paper_1805_08643_gb300.lbm import ERR_NONFINITE

    assert lat.check() in (ERR_EOS_DOMAIN, ERR_NONFINITE)
    assert lat.check() == OK
    lat.close()


def test_lagged_rejects_unsupported_forms():
    from paper_1805_08643_gb300.lbm import LBMError

    for grid, prec in (((25, 20, 28), "f32"), ((32, 32, 32), "f64")):
        lat = lattice(grid, "nonorth", prec, physics())
        with pytest.raises(LBMError, match="ERR_ARG"):
            lat.set_tuning("lagged")
        lat.close()
