"""Scheduling logic of the serving loop, on a fake backend (no GPU).

The fake backend mirrors the library's admission calls (prx_batch_admit by
device memory, prx_batch_step_epoch in whole reaction intervals that never
pass a job's step count, jobs with less than an interval left finishing
alone, prx_batch_poll) and advances a virtual clock by the work it is given,
so the checks are exact: every job takes exactly its steps, members only join
at the start of a reaction cycle, admitted memory never exceeds the budget,
admission follows arrival order when no job may go ahead of one that does not
fit (patience 0) and lets small jobs go ahead otherwise, and the latency
bookkeeping adds up.
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

    def __init__(self, clock, theta=10, budget=1 << 62):
        self.clock = clock
        self.theta = theta
        self.budget = budget
        self.used = 0
        self.members = {}  # slot -> system
        self.done = []
        self.log = []
        self.live = set()

    def estimate(self, job):
        return 1000 + 100 * job.n

    def fits(self, nbytes):
        return self.used + nbytes <= self.budget

    def create(self, job):
        h = dict(job=job, steps=0, left=None)
        self.live.add(id(h))
        self.clock.t += 1e-4
        return h

    def admit(self, h, nsteps):
        est = self.estimate(h["job"])
        if not self.fits(est):
            return None
        assert h["steps"] % self.theta == 0
        slot = 0
        while slot in self.members or slot in self.done:
            slot += 1
        self.members[slot] = h
        h["left"], h["est"] = nsteps, est
        self.used += est
        self.log.append(("admit", h["job"].job_id, h["steps"]))
        return slot

    def epoch(self, k):
        for slot, h in list(self.members.items()):  # finish alone
            if h["left"] < self.theta:
                h["steps"] += h["left"]
                self.clock.t += h["left"] * h["job"].n / self.RATE
                h["left"] = 0
                self.done.append(slot)
                del self.members[slot]
        if not self.members:
            return 0
        e = min(k, min(h["left"] for h in self.members.values()))
        if e >= self.theta:
            e -= e % self.theta
        assert e > 0
        for h in self.members.values():
            h["steps"] += e
            h["left"] -= e
        self.clock.t += e * sum(h["job"].n for h in self.members.values()) / self.RATE
        for slot, h in list(self.members.items()):
            if h["left"] == 0:
                self.done.append(slot)
                del self.members[slot]
        return e

    def poll(self):
        out, self.done = self.done, []
        return out

    def run_alone(self, h, k):
        h["steps"] += k
        self.clock.t += k * h["job"].n / self.RATE

    def finish(self, h):
        if "est" in h:
            self.used -= h["est"]
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
    budget = budget_jobs * (1000 + 100 * 262144)
    be = FakeBackend(clk, budget=budget)
    jobs = trace(7)
    srv = Server(be, budget, round_steps=200, theta=10, clock=clk, patience=0.0,
                 idle_wait=lambda: clk.sleep(1e-4))
    res = serve_trace(srv, jobs, clock=clk, sleep=clk.sleep)
    assert res["jobs"] == len(jobs) and len(srv.done) == len(jobs)
    for j in srv.done:
        assert j.result["steps"] == j.nsteps
        assert j.arrival <= j.admitted <= j.finished
    assert srv.peak_in_use <= budget and srv.in_use == 0 and be.used == 0
    assert not be.live  # every system freed
    # members join only at the start of a reaction cycle (fresh systems)
    assert all(steps == 0 for op, _, steps in be.log if op == "admit")
    # with no patience, admission is in arrival order
    adm = sorted(srv.done, key=lambda j: j.admitted)
    assert [j.job_id for j in adm] == sorted(j.job_id for j in jobs)
    if budget_jobs == 1:  # memory, not arrivals, held some jobs back
        assert any(j.admitted > j.arrival + 1e-3 for j in srv.done)
    if budget_jobs == 1000:
        assert srv.max_members > 3


def test_small_jobs_go_ahead_of_a_job_that_does_not_fit():
    """Backfilling: while a large job waits for memory, a later small job
    that fits is admitted; once the large job has waited longer than the
    patience, it holds the queue."""
    clk = FakeClock()
    big, small = 200_000, 2_000
    budget = (1000 + 100 * big) + (1000 + 100 * small) + 10
    be = FakeBackend(clk, budget=budget)
    jobs = [Job(job_id=0, nsteps=1000, arrival=0.0, system=None, n=big),
            Job(job_id=1, nsteps=50, arrival=0.001, system=None, n=big),
            Job(job_id=2, nsteps=50, arrival=0.002, system=None, n=small)]
    srv = Server(be, budget, round_steps=100, theta=10, clock=clk, patience=10.0,
                 idle_wait=lambda: clk.sleep(1e-4))
    serve_trace(srv, jobs, clock=clk, sleep=clk.sleep)
    by_id = {j.job_id: j for j in srv.done}
    assert by_id[2].admitted < by_id[1].admitted  # the small job went ahead
    assert all(j.result["steps"] == j.nsteps for j in srv.done)
    assert srv.peak_in_use <= budget


def test_batched_beats_serial_under_load_on_the_fake_clock():
    """With a backend whose batched step costs the same per particle as a
    single one, batching cannot lose throughput; it lowers latency by
    overlapping jobs (no head-of-line wait behind long jobs)."""
    clk = FakeClock()
    res_b = serve_trace(Server(FakeBackend(clk), 1 << 60, round_steps=100, clock=clk,
                               idle_wait=lambda: clk.sleep(1e-4)),
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
