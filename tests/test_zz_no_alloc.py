"""lbm_step_static: the step for callers that cannot allocate device memory.

Code running under CUDA-graph capture, or inside a host that owns all device
memory through its own allocator, cannot call cudaMalloc.  lbm_step_static
keeps its psi scratch in a static device array instead.  This test calls it
through the C ABI twice in a row (f0 -> f1 -> f2, device buffers from torch)
and compares each result with lbm_step's populations after the same number of
steps, within the FP64 parity tolerance of the other tests.  It sits in its
own file, collected last.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-11


@pytest.mark.parametrize("op", ["nonorth", "orth"])
def test_static_step_matches_lbm_step_on_two_calls(op):
    import torch

    from gpu_helpers import coexistence, lattice, physics
    from paper_1805_08643_gb300 import _build

    _build.build()
    from paper_1805_08643_gb300.lbm import ERR_ARG, OK, lib

    grid = (24, 20, 28)
    lat = lattice(grid, op, "f64", physics(sigma=0.105))
    rl, rv = coexistence(0.8)
    lat.init_droplet((12.0, 10.0, 14.0), 6.0, 2.0, rl, rv)
    f0 = torch.from_numpy(lat.populations()).cuda()
    f1 = torch.empty_like(f0)
    f2 = torch.empty_like(f0)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.lbm_step_static(lat.handle, ptr(f0), ptr(f1)) == OK
    assert lib.lbm_step_static(lat.handle, ptr(f1), ptr(f2)) == OK
    torch.cuda.synchronize()
    lat.step(1)
    ref1 = lat.populations()
    lat.step(1)
    ref2 = lat.populations()
    assert np.max(np.abs(f1.cpu().numpy() - ref1)) <= TOL_F64
    assert np.max(np.abs(f2.cpu().numpy() - ref2)) <= TOL_F64
    # aliasing and oversize boxes are rejected before any launch
    assert lib.lbm_step_static(lat.handle, ptr(f0), ptr(f0)) == ERR_ARG
    big = lattice((130, 128, 128), op, "f64", physics(), torch_buffers=False)
    assert lib.lbm_step_static(big.handle, ptr(f0), ptr(f1)) == ERR_ARG
    big.close()
    lat.close()
