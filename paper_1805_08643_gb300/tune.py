"""Autotuner of the batched step (work list or tile shape, z planes per work item) and of a single box's step.

Times a few steps of each candidate with CUDA events on the working stream and
keeps the fastest.  Results do not depend on the choice (tested), so tuning can
run on the live state: every candidate step is a real step of the simulation.
"""

from __future__ import annotations

TILES = {0: "32x4", 1: "32x8", 2: "64x4", 3: "work list (64x4 tile jobs)"}
WORK_LIST = 3


def _time(step, n, stream):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    step(n)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / n


def tune_batch(batch, tiles=(WORK_LIST, 0, 1, 2), z_planes=(16, 32, 64), steps=4):
    """Pick the batch's step kind (the work list, or a tile shape of the two-pass / single-pass kernels) and,
    for the latter, a common z-planes value; returns (tile, z, {candidate: ms/step})."""
    stream = batch.stream
    boxes = list(batch.grids)
    results = {}
    for t in tiles:
        for z in ((0,) if t == WORK_LIST else z_planes):
            for b in boxes:
                batch.set_tuning(t, b, z)
            batch.step(2)  # rebuild and warm the graph
            results[(t, z)] = _time(batch.step, steps, stream)
    best = min(results, key=results.get)
    for b in boxes:
        batch.set_tuning(best[0], b, best[1])
    return best[0], best[1], results


def tune_lattice(lat, tiles=(0, 1, 2), z_planes=(0, 16, 32, 64), steps=4):
    """Single box: compare the two-pass step with single-pass candidates; keep the fastest."""
    import torch

    stream = torch.cuda.current_stream()
    results = {}
    lat.set_tuning(False)
    lat.step(2)
    results[("two-pass",)] = _time(lat.step, steps, stream)
    for t in tiles:
        for z in z_planes:
            lat.set_tuning(True, t, z)
            lat.step(2)
            results[(t, z)] = _time(lat.step, steps, stream)
    best = min(results, key=results.get)
    if best == ("two-pass",):
        lat.set_tuning(False)
    else:
        lat.set_tuning(True, best[0], best[1])
    return best, results
