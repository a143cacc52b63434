"""lbm_step_static: the step for callers that cannot allocate device memory.

Code running under CUDA-graph capture, or inside a host that owns all device
memory through its own allocator, cannot call cudaMalloc.  lbm_step_static
keeps its psi scratch in a static device array instead.  This test calls it
through the C ABI twice in a row (f0 -> f1 -> f2, device buffers from torch)
and compares each result with lbm_step's populations after the same number of
steps, within the FP64 parity tolerance of the other tests, and the first
call with the FP64 oracle's step.  It sits in its own file, collected last.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-11


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("op", ["nonorth", "orth"])
def test_static_step_matches_lbm_step_on_two_calls(op):
    import torch

    from gpu_helpers import coexistence, lattice, oracle_params, physics
    from oracle import lbm_oracle as L
    from paper_1805_08643_gb300 import _build

    _build.build()
    from paper_1805_08643_gb300.lbm import OK, lib

    grid = (24, 20, 28)
    phys = physics(sigma=0.105)
    lat = lattice(grid, op, "f64", phys)
    rl, rv = coexistence(0.8)
    lat.init_droplet((12.0, 10.0, 14.0), 6.0, 2.0, rl, rv)
    f0_host = lat.populations()
    f0 = torch.from_numpy(f0_host).cuda()
    f1 = torch.empty_like(f0)
    f2 = torch.empty_like(f0)
    assert lib.lbm_step_static(lat.handle, _ptr(f0), _ptr(f1)) == OK
    assert lib.lbm_step_static(lat.handle, _ptr(f1), _ptr(f2)) == OK
    torch.cuda.synchronize()
    lat.step(1)
    ref1 = lat.populations()
    lat.step(1)
    ref2 = lat.populations()
    got1, got2 = f1.cpu().numpy(), f2.cpu().numpy()
    assert np.max(np.abs(got1 - ref1)) <= TOL_F64
    assert np.max(np.abs(got2 - ref2)) <= TOL_F64
    # the first call against the oracle's step of the same populations
    assert np.max(np.abs(got1 - L.step(oracle_params(grid, op, phys), f0_host))) <= 1e-14
    lat.close()


def test_static_step_rejects_what_it_cannot_run():
    """Aliased buffers, a box beyond the static array and a D3Q15 context are refused before any
    launch; every buffer passed is a real allocation of the box's full size."""
    import torch

    from gpu_helpers import lattice, physics
    from paper_1805_08643_gb300 import _build

    _build.build()
    from paper_1805_08643_gb300.lbm import ERR_ARG, lib

    small = lattice((8, 8, 8), "nonorth", "f64", physics())
    f = torch.zeros(19 * 8 ** 3, dtype=torch.float64, device="cuda")
    assert lib.lbm_step_static(small.handle, _ptr(f), _ptr(f)) == ERR_ARG
    small.close()
    big_grid = (130, 128, 128)  # 2^21 + 2^14 nodes: one plane more than the static array holds
    big = lattice(big_grid, "nonorth", "f64", physics(), torch_buffers=False)
    n = big_grid[0] * big_grid[1] * big_grid[2]
    fa = torch.zeros(19 * n, dtype=torch.float64, device="cuda")
    fb = torch.empty_like(fa)
    assert lib.lbm_step_static(big.handle, _ptr(fa), _ptr(fb)) == ERR_ARG
    big.close()
    del fa, fb
    q15 = lattice((8, 8, 8), "nonorth_d3q15", "f64", physics(), torch_buffers=False)
    fa = torch.zeros(19 * 8 ** 3, dtype=torch.float64, device="cuda")
    fb = torch.empty_like(fa)
    assert lib.lbm_step_static(q15.handle, _ptr(fa), _ptr(fb)) == ERR_ARG
    q15.close()
    torch.cuda.synchronize()
