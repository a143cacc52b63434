"""Scheduling logic of the job server, on the host with a fake backend."""

from paper_1805_08643_gb300.serve import Server
from paper_1805_08643_gb300.synth import JobSpec, job_stream


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeBackend:
    """Budgeted slots; each step costs time; a job converges after `need` steps."""

    def __init__(self, clock, budget, step_time=1e-4):
        self.clock, self.budget, self.used, self.step_time = clock, budget, 0, step_time
        self.live, self.next_id, self.admitted = {}, 0, []

    def bytes_for(self, spec):
        return spec.edge ** 3

    def admit(self, spec):
        if self.used + spec.edge ** 3 > self.budget:
            return None
        self.used += spec.edge ** 3
        box = self.next_id
        self.next_id += 1
        self.live[box] = [spec, 0]
        self.admitted.append(spec)
        return box

    def step(self, n):
        for v in self.live.values():
            v[1] += n
        self.clock.t += n * self.step_time
        assert self.used <= self.budget

    def max_du(self, boxes):
        # converges when steps >= 300 * edge / 48
        return [1e-9 if self.live[b][1] >= 300 * self.live[b][0].edge / 48 else 1.0 for b in boxes]

    def release(self, box):
        spec, _ = self.live.pop(box)
        self.used -= spec.edge ** 3


def test_every_job_finishes_within_budget_fifo():
    clock = FakeClock()
    jobs = job_stream(30, rate_per_s=200.0, edge_lo=48, edge_hi=96, seed=3)
    be = FakeBackend(clock, budget=3 * 96 ** 3)
    rep = Server(be, check_every=100, tol=1e-8, clock=clock, sleep=clock.sleep, keep_jobs=True).run(jobs)
    assert len(rep.latencies_s) == 30 and not be.live and be.used == 0
    assert [s.arrival for s in be.admitted] == sorted(s.arrival for s in jobs)  # FIFO admission
    assert rep.max_running <= 3 * 96 ** 3 // 48 ** 3
    for j in rep.jobs:
        assert j.steps == -(-int(300 * j.spec.edge / 48) // 100) * 100  # first check past convergence
        assert j.done_at >= j.spec.arrival
    s = rep.summary()
    assert s["p50_s"] <= s["p99_s"] and s["aggregate_mlups"] > 0
    assert rep.lattice_updates == sum(j.steps * j.spec.edge ** 3 for j in rep.jobs)


def test_max_steps_caps_a_job_that_never_converges():
    clock = FakeClock()
    be = FakeBackend(clock, budget=10 ** 9)
    be.max_du = lambda boxes: [1.0] * len(boxes)
    rep = Server(be, check_every=100, max_steps=500, clock=clock, sleep=clock.sleep, keep_jobs=True).run(
        [JobSpec(0.0, 48, "droplet", 0.7, "nonorth")])
    assert rep.jobs[0].steps == 500


def test_jobs_arriving_later_join_running_ones():
    clock = FakeClock()
    be = FakeBackend(clock, budget=10 ** 9, step_time=1e-3)
    jobs = [JobSpec(0.0, 96, "flat", 0.7, "orth"), JobSpec(0.15, 48, "droplet", 0.8, "nonorth")]
    rep = Server(be, check_every=100, clock=clock, sleep=clock.sleep, keep_jobs=True).run(jobs)
    a, b = sorted(rep.jobs, key=lambda j: j.spec.arrival)
    assert b.admitted_at < a.done_at  # the second job ran while the first was still on the device


def test_truncated_jobs_are_reported_apart_from_converged_ones():
    """Jobs stopped at max_steps do not enter the convergence latencies."""
    clock = FakeClock()
    jobs = job_stream(12, rate_per_s=100.0, edge_lo=48, edge_hi=144, seed=5)
    be = FakeBackend(clock, budget=4 * 144 ** 3)
    # converge needs 300 * edge / 48 steps: edges above 64 need more than max_steps = 400
    rep = Server(be, check_every=100, tol=1e-8, max_steps=400, min_steps=200, clock=clock,
                 sleep=clock.sleep, keep_jobs=True).run(jobs)
    s = rep.summary()
    want_conv = sum(1 for j in jobs if 300 * j.edge / 48 <= 400)
    assert s["converged"] == want_conv and s["truncated"] == len(jobs) - want_conv and s["jobs"] == len(jobs)
    assert all(j.converged == (300 * j.spec.edge / 48 <= 400) for j in rep.jobs)
    assert all(st <= 400 for st in rep.converged_steps)
    assert s["p50_all_s"] is not None
