"""The serving loop on the GPU: jobs that arrive while others run are admitted as memory
frees up, and every job's result is the same as the job run alone."""
import numpy as np
import pytest

from paper_2103_07925_gb300 import scenes as S
from paper_2103_07925_gb300.serve import Job, Server, poisson_arrivals

pytestmark = pytest.mark.gpu


def _jobs():
    arr = poisson_arrivals(8, 200.0, seed=7)
    specs = [S.tank2d_discs(dx=0.03, n_discs=3, seed=1), S.periodic_box(dim=3, n=10, bodies=1),
             S.tank3d_spheres(dx=0.06, n_spheres=2, r_range=(0.1, 0.12), size=(1.0, 1.0, 1.2), fill=0.6),
             S.periodic_box(dim=2, n=24, bodies=2, body_radius=0.2), S.tank2d_discs(dx=0.04, n_discs=0, seed=2),
             S.hydrostatic_tank2d(), S.cluster(dim=3, n=8), S.tank2d_discs(dx=0.025, n_discs=5, seed=3)]
    return [Job(q, sc, 5 + 3 * q, float(arr[q])) for q, sc in enumerate(specs)]


def _alone(job):
    from paper_2103_07925_gb300.sph import Scene
    g = Scene(job.scene, precision=32)
    g.step(job.steps)
    out = g.read("pos", "vel", "rho")
    g.close()
    return out


@pytest.mark.parametrize("cap_jobs", [None, 2])
def test_served_results_equal_alone(cap_jobs):
    from paper_2103_07925_gb300.sph import Batch
    jobs = _jobs()
    if cap_jobs is None:
        cap = 150 << 30
    else:  # memory for about two of the largest jobs: admissions wait for departures
        cap = cap_jobs * max(Batch.footprint(j.scene, precision=32) for j in jobs)
    B = Batch(capacity=16, hbm_cap_bytes=cap, precision=32)
    srv = Server(B, step_batch=4, fields=("pos", "vel", "rho"))
    done = srv.run(jobs)
    assert sorted(d.job_id for d in done) == list(range(len(jobs)))
    assert srv.max_bytes <= cap
    if cap_jobs is not None:
        assert srv.max_jobs < len(jobs)
    for d in done:
        ref = _alone(jobs[d.job_id])
        for f in ("pos", "vel", "rho"):
            np.testing.assert_array_equal(d.result[f], ref[f], err_msg="job %d %s" % (d.job_id, f))
    B.close()
