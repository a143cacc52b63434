"""Batched boxes (persistent launches over a work-item table, CUDA graphs) and continuous batching.

A batch whose boxes all have an even Nx steps on the two-pass pair kernels; one
box with an odd Nx puts the whole batch on the single-pass kernel.  Both are
compared with single-box runs.
"""

import numpy as np
import pytest

from gpu_helpers import coexistence, droplet_rho, lattice, max_abs, oracle_params, physics
from oracle import lbm_oracle as L

pytestmark = pytest.mark.gpu

BOXES = [  # grid, operator, T/T_c, sigma, W
    ((32, 32, 32), "nonorth", 0.8, 0.0, 2.0),
    ((24, 20, 28), "orth", 0.8, 0.105, 2.0),
    ((48, 40, 36), "nonorth", 0.7, 0.105, 5.0),
    ((36, 36, 40), "orth", 0.75, 0.0, 4.0),
]


def _add(batch, spec, prec="f32"):
    grid, op, t, sigma, W = spec
    phys = physics(T_over_Tc=t, sigma=sigma)
    from paper_1805_08643_gb300.lbm import Rates

    rates = Rates(phys["s_e"], phys["s_nu"], phys["s_q"], phys["s_pi"], phys["s_eps"], phys["s_m"])
    box = batch.add(grid, op, a=phys["a"], b=phys["b"], R=phys["R"], T=phys["T"], G=phys["G"], rates=rates,
                    sigma=sigma)
    rl, rv = coexistence(t)
    batch.init_droplet(box, tuple(n / 2 for n in grid), min(grid) / 4, W, rl, rv)
    return box


def _single(spec, steps, prec="f32"):
    grid, op, t, sigma, W = spec
    lat = lattice(grid, op, prec, physics(T_over_Tc=t, sigma=sigma))
    lat.set_tuning(True, 1, 0)
    rl, rv = coexistence(t)
    lat.init_droplet(tuple(n / 2 for n in grid), min(grid) / 4, W, rl, rv)
    lat.step(steps)
    out = lat.moments()
    lat.close()
    return out


def _batch(prec="f32", budget=1 << 36):
    from paper_1805_08643_gb300 import _build

    _build.build()
    from paper_1805_08643_gb300.lbm import Batch

    return Batch(prec, "cs", budget)


@pytest.mark.parametrize("steps", [20, 21])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_batch_matches_single_box_runs(steps, prec):
    b = _batch(prec)
    ids = [_add(b, s, prec) for s in BOXES]
    b.step(steps)
    assert b.check() == 0
    for box, spec in zip(ids, BOXES):
        rho, u = b.moments(box)
        rho1, u1 = _single(spec, steps, prec)
        # Separate kernel instantiations may contract FMAs differently: a last-bit FP32
        # difference, which FP16 storage turns into a flip of one half-precision ulp.
        tol = 1e-6 if prec == "f32" else 2e-3
        assert max_abs(rho, rho1) <= tol and max_abs(u, u1) <= tol, spec
        assert b.box_steps(box) == steps
    b.close()


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_batch_with_an_odd_nx_box_uses_the_single_pass_kernel(prec):
    boxes = [((25, 20, 28), "orth", 0.8, 0.105, 2.0), BOXES[0]]
    b = _batch(prec)
    ids = [_add(b, s, prec) for s in boxes]
    b.step(21)
    assert b.check() == 0
    for box, spec in zip(ids, boxes):
        rho, u = b.moments(box)
        rho1, u1 = _single(spec, 21, prec)
        tol = 1e-6 if prec == "f32" else 2e-3
        assert max_abs(rho, rho1) <= tol and max_abs(u, u1) <= tol, spec
    b.close()


def test_box_alone_equals_box_in_the_mix():
    alone = _batch()
    x = _add(alone, BOXES[2])
    alone.step(16)
    ref = alone.moments(x)
    alone.close()
    mix = _batch()
    ids = [_add(mix, s) for s in BOXES]
    mix.step(16)
    got = mix.moments(ids[2])
    mix.close()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_continuous_batching_join_and_leave():
    """A box that joins a running batch, while another leaves, evolves as if alone."""
    alone = _batch()
    q = _add(alone, BOXES[1])
    alone.step(14)
    ref = alone.moments(q)
    alone.close()

    b = _batch()
    p = _add(b, BOXES[0])
    b.step(10)
    q = _add(b, BOXES[1])  # joins after 10 steps
    b.step(10)
    b.remove(p)  # leaves
    r = _add(b, BOXES[3])  # another joins in the freed slot
    b.step(4)
    assert b.box_steps(q) == 14 and b.box_steps(r) == 4
    got = b.moments(q)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    b.close()


def test_admission_by_hbm_budget():
    from paper_1805_08643_gb300.lbm import Batch

    per_box = Batch.box_bytes("f32", BOXES[0][0])
    b = _batch(budget=2 * per_box + 1000)
    assert _add(b, BOXES[0]) is not None
    second = b.try_add(BOXES[0][0], "nonorth", T=0.07)
    assert second is not None
    assert b.try_add(BOXES[0][0], "nonorth", T=0.07) is None  # over budget: refused, not allocated
    assert b.info()["bytes_used"] == 2 * per_box
    b.remove(second)
    assert b.try_add(BOXES[0][0], "nonorth", T=0.07) is not None
    b.close()


def test_batch_box_against_fp64_oracle():
    spec = ((24, 20, 28), "orth", 0.8, 0.0, 2.0)
    b = _batch()
    box = _add(b, spec)
    b.step(200)
    rho, u = b.moments(box)
    b.close()
    grid = spec[0]
    phys = physics(T_over_Tc=0.8)
    rl, rv = coexistence(0.8)
    p = oracle_params(grid, "orth", phys)
    f = L.run(p, L.equilibrium_state(p, droplet_rho(grid, tuple(n / 2 for n in grid), min(grid) / 4, 2.0, rl, rv)), 200)
    rho_o, u_o, _, _ = L.macroscopic(p, f)
    assert max_abs(rho, rho_o) <= 2e-5 and max_abs(u, u_o) <= 2e-5


def test_max_du_tracks_convergence():
    b = _batch()
    box = _add(b, BOXES[0])
    d0 = b.max_du([box])[0]  # against u_prev = 0: the initial max |u|
    rho, u = b.moments(box)
    assert abs(d0 - float(np.sqrt((u * u).sum(0)).max())) < 1e-6
    b.step(100)
    d1 = b.max_du([box])[0]
    b.step(100)
    d2 = b.max_du([box])[0]
    assert d1 > 0 and d2 > 0 and d2 < d1  # a static droplet relaxes
    b.close()


def test_odd_step_counts_neither_rebuild_nor_change_the_result():
    """1 + 1 steps equal 2 steps bit for bit, and stepping one at a time recaptures nothing
    (the batch keeps a graph per starting parity)."""
    results = []
    for chunks in ([2], [1, 1], [1, 2, 1, 1, 3]):
        b = _batch()
        ids = [_add(b, s) for s in BOXES[:2]]
        b.step(chunks[0])
        builds = b.info()["graph_builds"]
        for n in chunks[1:]:
            b.step(n)
        assert b.info()["graph_builds"] == builds, chunks
        total = sum(chunks)
        assert all(b.box_steps(i) == total for i in ids)
        results.append((total, [b.moments(i) for i in ids]))
        b.close()
    (t0, r0), (t1, r1), _ = results
    assert t0 == t1 == 2
    for (a_rho, a_u), (b_rho, b_u) in zip(r0, r1):
        assert np.array_equal(a_rho, b_rho) and np.array_equal(a_u, b_u)


def _single_two_pass(spec, steps, prec):
    grid, op, t, sigma, W = spec
    lat = lattice(grid, op, prec, physics(T_over_Tc=t, sigma=sigma))
    lat.set_tuning(False)
    rl, rv = coexistence(t)
    lat.init_droplet(tuple(n / 2 for n in grid), min(grid) / 4, W, rl, rv)
    lat.step(steps)
    out = lat.moments()
    lat.close()
    return out


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_work_list_batch_equals_two_pass_batch(prec):
    """The batch's default step (the work list over all boxes, one launch per step) against the two-pass
    pair kernels over an odd and an even number of steps: equal bit for bit in FP32.  With FP16 storage
    the two-pass batch kernel can differ from single-box runs by one half-precision ulp (see above); the
    work list equals the single-box two-pass step bit for bit there."""
    outs = []
    for tile in (3, 1):
        b = _batch(prec)
        ids = [_add(b, s, prec) for s in BOXES]
        b.set_tuning(tile)
        b.step(7)
        b.step(6)
        assert b.check() == 0
        outs.append([b.moments(i) for i in ids])
        b.close()
    for spec, (r0, u0), (r1, u1) in zip(BOXES, *outs):
        if prec == "f32":
            assert np.array_equal(r0, r1) and np.array_equal(u0, u1), spec
        else:
            assert max_abs(r0, r1) <= 2e-3 and max_abs(u0, u1) <= 2e-3, spec
            rs, us = _single_two_pass(spec, 13, prec)
            assert np.array_equal(r0, rs) and np.array_equal(u0, us), spec


def test_work_list_batch_against_the_oracle_and_join_leave():
    """A box that joins a running work-list batch while another leaves evolves as the FP64 oracle says
    (FP32 tolerance), and the descriptors' counter bases follow the rebuilt list."""
    grid, op, t, sigma, W = BOXES[1]
    phys = physics(T_over_Tc=t, sigma=sigma)
    rl, rv = coexistence(t)
    b = _batch()
    p = _add(b, BOXES[0])
    b.step(5)
    q = _add(b, BOXES[1])
    b.step(3)
    b.remove(p)
    _add(b, BOXES[3])
    b.step(9)
    assert b.check() == 0
    rho, u = b.moments(q)
    b.close()
    po = oracle_params(grid, op, phys)
    centre = tuple(n / 2 for n in grid)
    f0 = L.equilibrium_state(po, droplet_rho(grid, centre, min(grid) / 4, W, rl, rv))
    rho_o, u_o, _, _ = L.macroscopic(po, L.run(po, f0, 12))
    assert max_abs(rho, rho_o) <= 2e-5 and max_abs(u, u_o) <= 2e-5


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_odd_and_even_boxes_in_one_batch_each_step_as_alone(prec):
    """A batch holding odd- and even-Nx boxes steps the even ones on the work list and the odd ones on the
    one-node single pass, in one graph: each box's result equals the box stepped alone, bit for bit."""
    mix = [((25, 20, 28), "orth", 0.8, 0.105, 2.0), BOXES[0], ((33, 30, 26), "nonorth", 0.75, 0.0, 3.0), BOXES[2]]
    b = _batch(prec)
    ids = [_add(b, s, prec) for s in mix]
    b.step(9)
    assert b.check() == 0
    got = [b.moments(i) for i in ids]
    b.close()
    for spec, (r, u) in zip(mix, got):
        alone = _batch(prec)
        i = _add(alone, spec, prec)
        alone.step(9)
        r1, u1 = alone.moments(i)
        alone.close()
        assert np.array_equal(r, r1) and np.array_equal(u, u1), spec
