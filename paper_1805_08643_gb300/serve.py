"""Continuous-batching job server for droplet and flat-interface runs.

Jobs (a box size, a droplet or a liquid slab, a reduced temperature, an
operator) arrive over time.  The server keeps every admitted job's populations
resident on the device inside one batch (include/lbm.h, "batches"), admits a
waiting job as soon as the batch's HBM budget has room for it, advances all
running jobs together (one step graph per check interval), and retires a job
when its velocity field has converged: max |u(t) - u(t - check_every)| below
``tol``, or when it reaches ``max_steps`` (reported apart, as truncated).
Latency is arrival to retirement.

The scheduling logic is independent of the device: ``Server`` drives any
backend with the ``BatchBackend`` interface, which the tests replace with a
host-only fake.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

from .synth import JobSpec

A_SERVE, B_SERVE, R_SERVE, G_SERVE = 0.25, 4.0, 1.0, -1.0
SIGMA_DROPLET, SIGMA_FLAT, W_DROPLET, W_FLAT = 0.105, 0.116, 5.0, 5.0


@dataclass
class JobState:
    spec: JobSpec
    job_id: int
    box: int | None = None
    admitted_at: float | None = None
    done_at: float | None = None
    steps: int = 0
    last_du: float | None = None
    converged: bool | None = None  # at retirement: converged, or stopped at max_steps


class BatchBackend:
    """Adapter from the server to ``lbm.Batch`` (one device, FP32 arithmetic)."""

    def __init__(self, precision="f32", hbm_budget_bytes=64 << 30):
        from . import thermo
        from .lbm import Batch, Rates

        self._thermo = thermo
        self._rates = Rates()
        self.batch = Batch(precision, "cs", hbm_budget_bytes)
        self.precision = precision

    def bytes_for(self, spec: JobSpec) -> int:
        return self.batch.box_bytes(self.precision, (spec.edge,) * 3)

    def admit(self, spec: JobSpec):
        """Add and initialise the job's box; None when the budget has no room."""
        th = self._thermo
        Tc = th.critical_temperature(A_SERVE, B_SERVE, R_SERVE)
        droplet = spec.kind == "droplet"
        box = self.batch.try_add((spec.edge,) * 3, spec.operator, a=A_SERVE, b=B_SERVE, R=R_SERVE,
                                 T=spec.T_over_Tc * Tc, G=G_SERVE, rates=self._rates,
                                 sigma=SIGMA_DROPLET if droplet else SIGMA_FLAT)
        if box is None:
            return None
        rl, rv = th.coexistence_cs(spec.T_over_Tc, A_SERVE, B_SERVE, R_SERVE)
        e = spec.edge
        if droplet:
            self.batch.init_droplet(box, (e / 2,) * 3, e / 4, W_DROPLET, rl, rv)
        else:
            self.batch.init_flat(box, 2, e / 4, 3 * e / 4, W_FLAT, rl, rv)
        return box

    def step(self, n: int):
        self.batch.step(n)

    def max_du(self, boxes):
        return self.batch.max_du(boxes)

    def release(self, box):
        self.batch.remove(box)

    def moments(self, box):
        return self.batch.moments(box)

    def close(self):
        self.batch.close()


def _percentile(values, q):
    if not values:
        return None
    xs = sorted(values)
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


@dataclass
class ServeReport:
    latencies_s: list = field(default_factory=list)            # jobs that converged
    truncated_latencies_s: list = field(default_factory=list)  # jobs retired at max_steps
    converged_steps: list = field(default_factory=list)
    lattice_updates: int = 0
    wall_s: float = 0.0
    max_running: int = 0
    jobs: list = field(default_factory=list)

    def percentile(self, q):
        """Arrival-to-convergence latency percentile over the converged jobs."""
        return _percentile(self.latencies_s, q)

    def summary(self):
        both = self.latencies_s + self.truncated_latencies_s
        steps = self.converged_steps
        return {"jobs": len(both), "converged": len(self.latencies_s),
                "truncated": len(self.truncated_latencies_s),
                "p50_s": self.percentile(50), "p99_s": self.percentile(99),
                "p50_all_s": _percentile(both, 50), "p99_all_s": _percentile(both, 99),
                "mean_steps_to_converge": sum(steps) / len(steps) if steps else None,
                "aggregate_mlups": self.lattice_updates / self.wall_s / 1e6 if self.wall_s > 0 else None,
                "wall_s": self.wall_s, "max_running": self.max_running}


class Server:
    """Admit-as-room-frees scheduler over one batch (continuous batching)."""

    def __init__(self, backend, check_every=100, tol=1e-8, max_steps=100_000, min_steps=200,
                 clock=time.perf_counter, sleep=time.sleep, keep_jobs=False):
        self.backend = backend
        self.check_every = check_every
        self.tol = tol
        self.max_steps = max_steps
        self.min_steps = min_steps
        self.clock = clock
        self.sleep = sleep
        self.keep_jobs = keep_jobs

    def run(self, jobs: list[JobSpec], on_retire=None) -> ServeReport:
        """Serve ``jobs`` (arrival times relative to the start) to completion."""
        pending = sorted((JobState(s, k) for k, s in enumerate(jobs)), key=lambda j: j.spec.arrival)
        waiting: list[JobState] = []
        running: list[JobState] = []
        report = ServeReport()
        t0 = self.clock()
        while pending or waiting or running:
            now = self.clock() - t0
            while pending and pending[0].spec.arrival <= now:
                waiting.append(pending.pop(0))
            # admit in arrival order while the budget has room
            still = []
            for j in waiting:
                box = self.backend.admit(j.spec) if not still else None
                if box is None:
                    still.append(j)
                else:
                    j.box, j.admitted_at = box, now
                    running.append(j)
            waiting = still
            report.max_running = max(report.max_running, len(running))
            if not running:
                if pending:
                    self.sleep(max(0.0, pending[0].spec.arrival - (self.clock() - t0)))
                continue
            self.backend.step(self.check_every)
            for j in running:
                j.steps += self.check_every
                report.lattice_updates += self.check_every * j.spec.edge ** 3
            du = self.backend.max_du([j.box for j in running])
            now = self.clock() - t0
            keep = []
            for j, d in zip(running, du):
                j.last_du = d
                converged = j.steps >= self.min_steps and d < self.tol
                if converged or j.steps >= self.max_steps:
                    j.done_at = now
                    j.converged = converged
                    if converged:
                        report.latencies_s.append(now - j.spec.arrival)
                        report.converged_steps.append(j.steps)
                    else:
                        report.truncated_latencies_s.append(now - j.spec.arrival)
                    if on_retire:
                        on_retire(j)
                    self.backend.release(j.box)
                    if self.keep_jobs:
                        report.jobs.append(j)
                else:
                    keep.append(j)
            running = keep
        report.wall_s = self.clock() - t0
        return report
