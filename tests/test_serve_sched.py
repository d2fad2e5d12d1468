"""Scheduling logic of the serving loop, on a fake backend (no GPU).

The fake backend keeps, per system, the steps it has taken and whether it is
in the batch, and advances a virtual clock by the work it is given, so the
checks are exact: every job takes exactly its steps, members only join at the
start of a reaction cycle, admitted memory never exceeds the budget,
admission follows arrival order, and the latency bookkeeping adds up.
"""
import numpy as np
import pytest

from paper_1409_7498_gb300.serve import Job, Server, serve_serial, serve_trace


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeBackend:
    RATE = 1e9  # particle-steps per second of virtual time

    def __init__(self, clock, theta=10):
        self.clock = clock
        self.theta = theta
        self.members = []
        self.log = []
        self.live = set()

    def estimate(self, job):
        return 1000 + 100 * job.n

    def create(self, job):
        h = dict(job=job, steps=0, in_batch=False)
        self.live.add(id(h))
        self.clock.t += 1e-4
        return h

    def add(self, h):
        assert not h["in_batch"] and h["steps"] % self.theta == 0
        h["in_batch"] = True
        self.members.append(h)
        self.log.append(("add", h["job"].job_id, h["steps"]))

    def remove(self, h):
        assert h["in_batch"]
        h["in_batch"] = False
        self.members.remove(h)

    def run(self, k):
        assert k > 0 and k % self.theta == 0 and self.members
        for h in self.members:
            h["steps"] += k
        self.clock.t += k * sum(h["job"].n for h in self.members) / self.RATE

    def sync(self):
        pass

    def run_alone(self, h, k):
        assert not h["in_batch"]
        h["steps"] += k
        self.clock.t += k * h["job"].n / self.RATE

    def finish(self, h):
        return dict(steps=h["steps"])

    def close(self, h):
        self.live.discard(id(h))


def trace(seed, count=60, rate=20.0):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    n = np.exp(rng.uniform(np.log(2048), np.log(262144), count)).astype(int)
    steps = np.exp(rng.uniform(np.log(5), np.log(5000), count)).astype(int)
    return [Job(job_id=i, nsteps=int(steps[i]), arrival=float(t[i]), system=None, n=int(n[i]))
            for i in range(count)]


@pytest.mark.parametrize("budget_jobs", [1, 3, 1000])
def test_every_job_runs_exactly_its_steps(budget_jobs):
    clk = FakeClock()
    be = FakeBackend(clk)
    jobs = trace(7)
    budget = budget_jobs * (1000 + 100 * 262144)
    srv = Server(be, budget, round_steps=200, theta=10, clock=clk)
    res = serve_trace(srv, jobs, clock=clk, sleep=clk.sleep)
    assert res["jobs"] == len(jobs) and len(srv.done) == len(jobs)
    for j in srv.done:
        assert j.result["steps"] == j.nsteps
        assert j.arrival <= j.admitted <= j.finished
    assert srv.peak_in_use <= budget and srv.in_use == 0
    assert not be.live  # every system freed
    # members join only at the start of a reaction cycle (fresh systems)
    assert all(steps == 0 for op, _, steps in be.log if op == "add")
    # admission in arrival order
    adm = sorted(srv.done, key=lambda j: j.admitted)
    assert [j.job_id for j in adm] == sorted(j.job_id for j in jobs)
    if budget_jobs == 1:  # memory, not arrivals, held some jobs back
        assert any(j.admitted > j.arrival + 1e-3 for j in srv.done)
    if budget_jobs == 1000:
        assert srv.max_members > 3


def test_batched_beats_serial_under_load_on_the_fake_clock():
    """With a backend whose batched step costs the same per particle as a
    single one, batching cannot lose throughput; it lowers latency by
    overlapping jobs (no head-of-line wait behind long jobs)."""
    clk = FakeClock()
    res_b = serve_trace(Server(FakeBackend(clk), 1 << 60, round_steps=100, clock=clk),
                        trace(3, 40, rate=200.0), clock=clk, sleep=clk.sleep)
    clk2 = FakeClock()
    res_s = serve_serial(FakeBackend(clk2), trace(3, 40, rate=200.0), clock=clk2, sleep=clk2.sleep)
    assert res_b["jobs"] == res_s["jobs"] == 40
    assert res_b["p50_latency_s"] <= res_s["p50_latency_s"]


def test_job_larger_than_the_budget_is_refused():
    clk = FakeClock()
    srv = Server(FakeBackend(clk), 5000, clock=clk)
    with pytest.raises(ValueError):
        srv.submit(Job(job_id=0, nsteps=10, arrival=0.0, system=None, n=1000))


def test_round_steps_must_be_whole_intervals():
    with pytest.raises(ValueError):
        Server(FakeBackend(FakeClock()), 1 << 30, round_steps=25, theta=10)
