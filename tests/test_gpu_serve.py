"""The job server on the GPU: results do not depend on what else was running."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_each_served_result_equals_the_job_run_alone():
    from paper_1805_08643_gb300 import _build

    _build.build()
    from paper_1805_08643_gb300.serve import BatchBackend, Server
    from paper_1805_08643_gb300.synth import JobSpec

    jobs = [JobSpec(0.00, 24, "droplet", 0.7, "nonorth"), JobSpec(0.00, 32, "flat", 0.8, "orth"),
            JobSpec(0.02, 28, "droplet", 0.65, "orth"), JobSpec(0.05, 36, "flat", 0.75, "nonorth"),
            JobSpec(0.05, 24, "droplet", 0.9, "orth")]
    served = {}
    be = BatchBackend("f32", hbm_budget_bytes=1 << 40)
    server = Server(be, check_every=100, tol=1e-6, max_steps=600, min_steps=200, keep_jobs=True)
    rep = server.run(jobs, on_retire=lambda j: served.__setitem__(j.job_id, (j.steps, be.moments(j.box))))
    be.close()
    assert len(served) == len(jobs) and rep.max_running >= 2
    for k, spec in enumerate(jobs):
        steps, (rho, u) = served[k]
        alone = BatchBackend("f32")
        box = alone.admit(spec)
        alone.step(steps)
        rho1, u1 = alone.moments(box)
        alone.close()
        assert np.array_equal(rho, rho1) and np.array_equal(u, u1), (k, spec)


def test_admission_waits_for_room():
    from paper_1805_08643_gb300.lbm import Batch
    from paper_1805_08643_gb300.serve import BatchBackend, Server
    from paper_1805_08643_gb300.synth import JobSpec

    per = Batch.box_bytes("f32", (32, 32, 32))
    be = BatchBackend("f32", hbm_budget_bytes=2 * per)
    jobs = [JobSpec(0.0, 32, "droplet", 0.8, "nonorth") for _ in range(5)]
    rep = Server(be, check_every=100, tol=0.0, max_steps=200, keep_jobs=True).run(jobs)
    be.close()
    s = rep.summary()  # tol = 0: every job stops at max_steps and counts as truncated
    assert s["jobs"] == 5 and s["truncated"] == 5 and s["converged"] == 0 and rep.max_running == 2
