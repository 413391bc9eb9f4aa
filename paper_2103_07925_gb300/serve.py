"""Serving loop: scene jobs arrive over time, are admitted into a resident batch while their
device footprint fits under a memory cap, advance together in step batches, and leave when
they reach their step count (continuous batching).  The plain path serves the same arrival
sequence one scene at a time.

The loop is host logic only: admission, stepping and polling go through the batch calls of
libsph (sph_batch_admit / sph_batch_step / sph_batch_poll), which copy the job's inputs to
the device, keep its state resident and run every stage of a step as one launch over all
resident scenes.  Any object with the methods of ``sph.Batch`` serves (the CPU tests use a
fake one).
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    job_id: int            # caller's id
    scene: dict            # scene dictionary (host inputs)
    steps: int             # steps to run
    arrival: float         # seconds after the start of the run
    overrides: dict = field(default_factory=dict)


@dataclass
class Done:
    job_id: int
    arrival: float
    admitted: float
    finished: float
    result: dict
    failed: bool = False   # velocities became non-finite; the job stopped early

    @property
    def latency(self):
        return self.finished - self.arrival


def poisson_arrivals(n, rate, seed=2103):
    """n arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def percentiles(done):
    lat = np.array([d.latency for d in done])
    if lat.size == 0:
        return dict(p50=float("nan"), p99=float("nan"), mean=float("nan"))
    return dict(p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99)), mean=float(lat.mean()))


def job_work(j):
    """Particle-steps of a job (its cost on the device, up to a per-step overhead)."""
    return len(j.scene["particles"]["mass"]) * j.steps if "particles" in j.scene else j.scene["n"] * j.steps


def job_particles(j):
    return len(j.scene["particles"]["mass"]) if "particles" in j.scene else j.scene["n"]


class Server:
    """Continuous batching of scene jobs on one GPU.

    Every resident job advances by one step per batch step, so a job's latency is its step
    count times the duration of the batch steps it shares.  Two admission policies:

    * ``fifo``: arrival order; the head of the queue is admitted as soon as a slot is free
      and its footprint fits under the cap (no overtaking).
    * ``sjf``: among the jobs that have arrived, the one with the least work (particles x
      steps) first, while the resident particles stay within ``max_particles`` (a job larger
      than the budget runs when the batch is otherwise empty).  A job that has waited longer
      than ``max_wait`` seconds goes first, so that large jobs are not starved.

    While jobs are resident the batch advances by ``step_batch`` steps per iteration;
    finished jobs are read out (``fields``) and released, which frees their slot and memory.
    """

    def __init__(self, batch, step_batch=10, fields=("pos", "vel"), policy="fifo", max_particles=None,
                 max_wait=float("inf"), clock=time.perf_counter, sleep=time.sleep):
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be fifo or sjf")
        self.batch = batch
        self.step_batch = step_batch
        self.fields = tuple(fields)
        self.policy = policy
        self.max_particles = max_particles
        self.max_wait = max_wait
        self.clock = clock
        self.sleep = sleep
        self.max_bytes = 0
        self.max_jobs = 0

    def _pick(self, arrived, t):
        """Index in ``arrived`` of the next job to admit."""
        if self.policy == "fifo":
            return 0
        late = [q for q, j in enumerate(arrived) if t - j.arrival > self.max_wait]
        if late:
            return late[0]
        return min(range(len(arrived)), key=lambda q: (job_work(arrived[q]), arrived[q].arrival))

    def run(self, jobs):
        queue = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        arrived = []    # arrived, not admitted (arrival order)
        resident = {}   # batch id -> (job, admitted time)
        live = 0        # resident particles
        done = []
        t0 = self.clock()
        now = lambda: self.clock() - t0
        while queue or arrived or resident:
            t = now()
            while queue and queue[0].arrival <= t:
                arrived.append(queue.popleft())
            # admissions in policy order while they fit
            while arrived:
                q = self._pick(arrived, t)
                j = arrived[q]
                n = job_particles(j)
                if self.max_particles is not None and resident and live + n > self.max_particles:
                    break
                bid = self.batch.admit(j.scene, j.steps, **j.overrides)
                if bid is None:
                    if not resident:
                        raise RuntimeError("job %d does not fit into an empty batch" % j.job_id)
                    break
                arrived.pop(q)
                live += n
                resident[bid] = (j, now())
            info = self.batch.info()
            self.max_bytes = max(self.max_bytes, info["bytes"])
            self.max_jobs = max(self.max_jobs, info["jobs"])
            if not resident:
                # idle until the next arrival
                self.sleep(max(0.0, queue[0].arrival - now()))
                continue
            self.batch.step(self.step_batch)
            for bid in self.batch.poll():
                j, ta = resident.pop(bid)
                live -= job_particles(j)
                failed = self.batch.state(bid) == "failed" if hasattr(self.batch, "state") else False
                res = self.batch.read(bid, *self.fields) if self.fields else {}
                if len(self.fields) == 1:
                    res = {self.fields[0]: res}
                self.batch.release(bid)
                done.append(Done(j.job_id, j.arrival, ta, now(), res, failed))
        return done


def serve_plain(jobs, make_scene, fields=("pos", "vel"), policy="fifo", clock=time.perf_counter, sleep=time.sleep):
    """The same arrivals served one scene at a time: create, run all steps, read, destroy.
    ``policy`` picks the next job among those that have arrived (fifo or sjf, as above)."""
    done = []
    t0 = clock()
    now = lambda: clock() - t0
    queue = collections.deque(sorted(jobs, key=lambda j: j.arrival))
    arrived = []
    while queue or arrived:
        while queue and queue[0].arrival <= now():
            arrived.append(queue.popleft())
        if not arrived:
            sleep(max(0.0, queue[0].arrival - now()))
            continue
        q = 0 if policy == "fifo" else min(range(len(arrived)), key=lambda q: (job_work(arrived[q]), arrived[q].arrival))
        j = arrived.pop(q)
        ta = now()
        g = make_scene(j.scene, **j.overrides)
        failed = False
        try:
            g.step(j.steps)
        except RuntimeError as e:  # non-finite velocities end the job early, as in the batch
            if getattr(e, "status", None) != -4:
                raise
            failed = True
        res = g.read(*fields) if fields else {}
        if len(fields) == 1:
            res = {fields[0]: res}
        g.close()
        done.append(Done(j.job_id, j.arrival, ta, now(), res, failed))
    return done


def serving_jobs(count, rate=20.0, n_lo=5e3, n_hi=1e6, max_bodies=100, steps=1000, seed=2103, precision=32):
    """Jobs of the serving workload: N log-uniform in [n_lo, n_hi], 0..max_bodies bodies,
    2D or 3D by a seeded coin, Poisson arrivals at ``rate`` per second."""
    from . import scenes as S
    rng = np.random.default_rng(seed)
    arr = poisson_arrivals(count, rate, seed=seed + 1)
    jobs = []
    for q in range(count):
        n_t = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        dim = 2 if rng.uniform() < 0.5 else 3
        nb = int(rng.integers(0, max_bodies + 1))
        dx = S.dx_for_count(dim, n_t)
        s = int(rng.integers(0, 2 ** 31 - 1))
        if dim == 2:
            sc = S.tank2d_discs(dx=dx, n_discs=nb, seed=s, precision=precision)
        else:
            sc = S.tank3d_spheres(dx=dx, n_spheres=nb, seed=s, r_range=(max(0.04, 1.5 * dx), max(0.08, 2.0 * dx)),
                                  precision=precision, allow_fewer=True, max_tries=20000)
        jobs.append(Job(q, sc, steps, float(arr[q])))
    return jobs
