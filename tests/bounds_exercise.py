"""Run every step kind of the library on tiny boxes and print one JSON line of statuses and checksums.

Used by tests/test_gpu_bounds.py, once with the debug build of the library
(LBM_DEBUG_LIBRARY=1: kernel indices checked, lbm_check reports LBM_ERR_BOUNDS)
and once with the normal build.  Boxes: 4^3 and 6 x 5 x 7 (and 5 x 4 x 4 for the
odd-Nx paths), so that every periodic wrap is also a tile edge.
"""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402

from gpu_helpers import coexistence, lattice, physics  # noqa: E402

GRIDS = [(4, 4, 4), (6, 5, 7)]


def checksum(rho, u):
    return [float(np.sum(rho)), float(np.sum(np.abs(u))), float(np.max(rho)), float(np.min(rho))]


def run_box(grid, op, prec, mode, out):
    phys = physics(sigma=0.105 if op != "nonorth_d3q15" else 0.0)
    rl, rv = coexistence(0.8)
    lat = lattice(grid, op, prec, phys)
    if mode is not None:
        lat.set_tuning(mode, 1, 0)
    lat.init_droplet(tuple(n / 2 for n in grid), min(grid) / 3, 2.0, rl, rv)
    lat.step(3)
    st = [lat.check()]
    rho, u = lat.moments()
    f = lat.populations()
    lat.set_populations(f)
    lat.step(1)
    st.append(lat.check())
    d = lat.diag()
    st.append(lat.check())
    out[f"{op}/{prec}/{mode}/{grid}"] = {"status": st, "sum": checksum(rho, u), "mass": d["mass"]}
    lat.close()


def run_batch(prec, tile, boxes, out):
    from paper_1805_08643_gb300.lbm import Batch

    b = Batch(prec, "cs", 1 << 32)
    ids = []
    rl, rv = coexistence(0.8)
    for k, grid in enumerate(boxes):
        phys = physics(sigma=0.105)
        from paper_1805_08643_gb300.lbm import Rates

        box = b.add(grid, "nonorth" if k % 2 == 0 else "orth", a=phys["a"], b=phys["b"], R=phys["R"], T=phys["T"],
                    G=phys["G"], rates=Rates(), sigma=0.105)
        b.init_droplet(box, tuple(n / 2 for n in grid), min(grid) / 3, 2.0, rl, rv)
        ids.append(box)
    b.set_tuning(tile)
    b.step(3)
    st = [b.check()]
    sums = [checksum(*b.moments(i)) for i in ids]
    b.max_du(ids)
    st.append(b.check())
    out[f"batch/{prec}/{tile}/{boxes}"] = {"status": st, "sum": sums}
    b.close()


def main():
    import torch

    torch.cuda.set_device(0)
    out = {}
    for grid in GRIDS:
        for op in ("nonorth", "orth", "nonorth_d3q15"):
            for prec in ("f64", "f32", "f16"):
                run_box(grid, op, prec, None, out)
        for op in ("nonorth", "orth"):
            for mode in (False, True, "lagged", "queue", "onchip"):
                run_box(grid, op, "f32", mode, out)
            for mode in (True, "queue"):
                run_box(grid, op, "f16", mode, out)
        for prec in ("f32", "f16"):
            run_box(grid, "nonorth_d3q15", prec, "queue", out)
            run_box(grid, "nonorth_d3q15", prec, False, out)
    run_box((5, 4, 4), "nonorth", "f32", None, out)  # odd Nx: one-node kernels
    run_box((5, 4, 4), "orth", "f32", True, out)
    for prec in ("f32", "f16"):
        for tile in (3, 0, 1, 2):
            run_batch(prec, tile, [(6, 5, 7), (4, 4, 4), (8, 6, 5)], out)
        run_batch(prec, 1, [(5, 4, 4), (4, 4, 4)], out)  # an odd-Nx box: the one-node single pass
    # the no-alloc FP64 step on the public layout
    import ctypes

    from paper_1805_08643_gb300.lbm import lib

    lat = lattice((6, 5, 7), "nonorth", "f64", physics())
    rl, rv = coexistence(0.8)
    lat.init_droplet((3.0, 2.5, 3.5), 2.0, 2.0, rl, rv)
    f0 = torch.from_numpy(lat.populations()).cuda()
    f1 = torch.empty_like(f0)
    st = lib.lbm_step_static(lat.handle, ctypes.c_void_p(f0.data_ptr()), ctypes.c_void_p(f1.data_ptr()))
    torch.cuda.synchronize()
    out["static/f64"] = {"status": [st, lat.check()], "sum": [float(f1.sum())]}
    lat.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
