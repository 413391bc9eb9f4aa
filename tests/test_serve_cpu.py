"""Host logic of the serving loop against a fake batch and a fake clock (no GPU)."""
import numpy as np
import pytest

from paper_2103_07925_gb300.serve import Job, Server, percentiles, poisson_arrivals, serve_plain


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(0.0, dt)


class FakeBatch:
    """Footprint = 100 bytes per particle; a step costs 1 us per resident particle."""

    def __init__(self, clock, cap_bytes, capacity=8):
        self.clock, self.cap, self.capacity = clock, cap_bytes, capacity
        self.jobs = {}
        self.next = 0
        self.peak = 0
        self.order = []

    def admit(self, scene, steps, **kw):
        need = 100 * scene["n"]
        used = sum(100 * j["n"] for j in self.jobs.values())
        if len(self.jobs) >= self.capacity or used + need > self.cap:
            return None
        jid = self.next
        self.next += 1
        self.jobs[jid] = dict(n=scene["n"], left=steps, done=False, reported=False, name=scene["name"])
        self.order.append(scene["name"])
        self.peak = max(self.peak, used + need)
        return jid

    def step(self, k):
        while k > 0:
            act = [j for j in self.jobs.values() if not j["done"]]
            if not act:
                return
            c = min(k, min(j["left"] for j in act))
            self.clock.t += c * 1e-6 * sum(j["n"] for j in act)
            for j in act:
                j["left"] -= c
                j["done"] = j["left"] == 0
            k -= c

    def poll(self):
        out = [i for i, j in self.jobs.items() if j["done"] and not j["reported"]]
        for i in out:
            self.jobs[i]["reported"] = True
        return out

    def read(self, jid, *names):
        return {nm: self.jobs[jid]["name"] for nm in names} if len(names) > 1 else self.jobs[jid]["name"]

    def release(self, jid):
        del self.jobs[jid]

    def info(self):
        return dict(bytes=sum(100 * j["n"] for j in self.jobs.values()), jobs=len(self.jobs))


def _jobs(sizes, arrivals, steps=100):
    return [Job(q, dict(n=n, name="j%d" % q), steps, a) for q, (n, a) in enumerate(zip(sizes, arrivals))]


def test_all_jobs_finish_under_the_cap_in_arrival_order():
    clk = Clock()
    fb = FakeBatch(clk, cap_bytes=100 * 3000)
    jobs = _jobs([1000, 2000, 500, 1500, 800], [0.0, 0.01, 0.02, 0.03, 0.5])
    done = Server(fb, step_batch=10, clock=clk, sleep=clk.sleep).run(jobs)
    assert sorted(d.job_id for d in done) == list(range(5))
    assert fb.peak <= fb.cap
    assert fb.order == ["j0", "j1", "j2", "j3", "j4"]  # no overtaking
    for d in done:
        assert d.admitted >= d.arrival and d.finished > d.admitted
        assert d.result["pos"] == "j%d" % d.job_id


def test_large_job_waits_for_memory_and_small_ones_do_not_overtake():
    clk = Clock()
    fb = FakeBatch(clk, cap_bytes=100 * 2000)
    jobs = _jobs([1500, 1800, 100], [0.0, 0.0, 0.0])
    done = {d.job_id: d for d in Server(fb, step_batch=5, clock=clk, sleep=clk.sleep).run(jobs)}
    # job 1 is admitted only once job 0 has left; job 2 behind it waits too
    assert done[1].admitted >= done[0].finished
    assert done[2].admitted >= done[1].admitted


def test_job_that_never_fits_is_an_error():
    clk = Clock()
    fb = FakeBatch(clk, cap_bytes=100 * 100)
    with pytest.raises(RuntimeError):
        Server(fb, clock=clk, sleep=clk.sleep).run(_jobs([500], [0.0]))


def test_idle_server_waits_for_arrivals():
    clk = Clock()
    fb = FakeBatch(clk, cap_bytes=10 ** 9)
    done = Server(fb, clock=clk, sleep=clk.sleep).run(_jobs([10], [2.0], steps=10))
    assert done[0].admitted >= 2.0


def test_batching_beats_one_at_a_time_on_latency_when_work_overlaps():
    """With a cost model where a batched step of many small scenes costs less than their
    separate steps (launch overhead per step), the batched server has lower p50."""
    class OverheadBatch(FakeBatch):
        def step(self, k):
            while k > 0:
                act = [j for j in self.jobs.values() if not j["done"]]
                if not act:
                    return
                c = min(k, min(j["left"] for j in act))
                self.clock.t += c * (50e-6 + 1e-8 * sum(j["n"] for j in act))
                for j in act:
                    j["left"] -= c
                    j["done"] = j["left"] == 0
                k -= c

    class PlainScene:
        def __init__(self, clk, scene):
            self.clk, self.sc = clk, scene

        def step(self, k):
            self.clk.t += k * (50e-6 + 1e-8 * self.sc["n"])

        def read(self, *names):
            return self.sc["name"]

        def close(self):
            pass

    arr = poisson_arrivals(20, 200.0, seed=4)
    sizes = [1000] * 20
    clk = Clock()
    batched = Server(OverheadBatch(clk, 10 ** 9, capacity=32), clock=clk, sleep=clk.sleep).run(_jobs(sizes, arr, 500))
    clk2 = Clock()
    plain = serve_plain(_jobs(sizes, arr, 500), lambda sc: PlainScene(clk2, sc), fields=("pos",),
                        clock=clk2, sleep=clk2.sleep)
    assert percentiles(batched)["p50"] < percentiles(plain)["p50"]
    assert len(batched) == len(plain) == 20


def test_poisson_arrivals_have_the_requested_rate():
    a = poisson_arrivals(20000, 20.0, seed=1)
    assert np.all(np.diff(a) > 0)
    assert abs(len(a) / a[-1] - 20.0) < 0.5


def test_sjf_admits_least_work_first_within_the_particle_budget():
    clk = Clock()
    fb = FakeBatch(clk, cap_bytes=10 ** 12, capacity=64)
    sizes = [5000, 100, 3000, 200, 50]
    done = Server(fb, step_batch=10, policy="sjf", max_particles=3000, clock=clk, sleep=clk.sleep).run(
        _jobs(sizes, [0.0] * 5))
    assert fb.order[:3] == ["j4", "j1", "j3"]  # least work first
    assert len(done) == 5
    lat = {d.job_id: d.latency for d in done}
    assert lat[4] < lat[2] < lat[0]


def test_sjf_budget_is_respected_and_oversized_job_runs_alone():
    clk = Clock()

    class Watch(FakeBatch):
        peak_n = 0

        def step(self, k):
            live = sum(j["n"] for j in self.jobs.values() if not j["done"])
            Watch.peak_n = max(Watch.peak_n, live)
            super().step(k)

    fb = Watch(clk, cap_bytes=10 ** 12, capacity=64)
    done = Server(fb, step_batch=5, policy="sjf", max_particles=1000, clock=clk, sleep=clk.sleep).run(
        _jobs([400, 400, 400, 2500], [0.0, 0.0, 0.0, 0.0]))
    assert len(done) == 4
    assert Watch.peak_n == 2500  # the oversized job alone; the small ones at most 800 together


def test_sjf_aging_lets_a_large_job_through():
    clk = Clock()
    fb = FakeBatch(clk, cap_bytes=10 ** 12, capacity=64)
    # a stream of small jobs would starve the large one without aging
    sizes = [3000] + [100] * 30
    arr = [0.0] + [0.001 * q for q in range(30)]
    done = {d.job_id: d for d in Server(fb, step_batch=10, policy="sjf", max_particles=3000, max_wait=0.005,
                                        clock=clk, sleep=clk.sleep).run(_jobs(sizes, arr))}
    assert done[0].admitted < max(d.admitted for d in done.values())


def test_plain_sjf_serves_small_jobs_first():
    class PlainScene:
        def __init__(self, clk, scene):
            self.clk, self.sc = clk, scene

        def step(self, k):
            self.clk.t += k * 1e-6 * self.sc["n"]

        def read(self, *names):
            return self.sc["name"]

        def close(self):
            pass

    clk = Clock()
    done = serve_plain(_jobs([5000, 10, 20], [0.0, 0.0, 0.0]), lambda sc: PlainScene(clk, sc), fields=("pos",),
                       policy="sjf", clock=clk, sleep=clk.sleep)
    assert [d.job_id for d in done] == [1, 2, 0]
