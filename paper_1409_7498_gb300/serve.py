"""Serving loop: polymerisation jobs of different sizes arrive over time and
share one GPU through one prx_batch (continuous batching).

Each job is a system (positions, velocities, types, states, a reaction
scheme, a seed) and a number of MD steps.  The loop:

  * admits queued jobs in arrival order while their device-memory estimate
    (prx_estimate_bytes) fits the budget; an admitted job's system is created
    (uploaded and binned) while the batch is busy on the GPU;
  * runs the batch in rounds of whole reaction intervals, so that every
    member stays at the start of its reaction cycle between rounds and new
    jobs can join at any round;
  * a job with fewer steps left than one interval leaves the batch and runs
    its last steps alone (the same kernels on the same data: a job's result
    does not depend on which other jobs shared the GPU with it);
  * a finished job's bonds and states are read back, its memory freed, and
    its latency (arrival to result) recorded.

All simulation work runs in the library's CUDA kernels; this module only
schedules.  The backend interface is small so that the scheduling logic can
be tested without a GPU.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import Any, Callable, Optional

import numpy as np


@dataclasses.dataclass
class Job:
    """One request.  `system` holds what the backend needs to create the
    system (for polyrx: desc, pos, vel, type, state, reaction)."""
    job_id: int
    nsteps: int
    arrival: float
    system: Any
    n: int = 0
    est_bytes: int = 0
    admitted: Optional[float] = None
    finished: Optional[float] = None
    result: Any = None
    steps_done: int = 0
    handle: Any = None

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival


class PolyrxBackend:
    """Backend on the polyrx C ABI (prx_create / prx_batch_*)."""

    def __init__(self, P, stream=None, positions: bool = False):
        self.P = P
        self.batch = P.Batch(stream=stream)
        self.positions = positions

    def estimate(self, job: Job) -> int:
        return self.P.prx_estimate_bytes(job.system["desc"])

    def create(self, job: Job):
        s = job.system
        g = self.P.System(s["desc"], s["pos"], s.get("vel"), s["type"], s["state"])
        if s.get("reaction") is not None:
            g.set_reaction(s["reaction"])
        return g

    def add(self, h):
        self.batch.add(h)

    def remove(self, h):
        self.batch.remove(h)

    def run(self, nsteps: int):
        self.batch.run(nsteps)

    def sync(self):
        self.batch.sync()

    def run_alone(self, h, nsteps: int):
        h.run(nsteps)

    def finish(self, h):
        """Reads the job's result back (synchronises its stream)."""
        out = dict(bonds=h.bonds(), states=h.states(), step=h.step())
        if self.positions:
            out["positions"] = h.positions()
        return out

    def close(self, h):
        h.close()

    def shutdown(self):
        self.batch.close()


class Server:
    """Continuous-batching scheduler.

    mem_budget : device bytes the admitted jobs may occupy together
    round_steps: MD steps per batch round (a multiple of theta)
    theta      : the reaction interval shared by the jobs
    clock      : time source (seconds)
    """

    def __init__(self, backend, mem_budget: int, round_steps: int = 200, theta: int = 10,
                 clock: Callable[[], float] = time.perf_counter):
        if round_steps % theta:
            raise ValueError("round_steps must be a multiple of theta")
        self.be = backend
        self.budget = int(mem_budget)
        self.round_steps = round_steps
        self.theta = theta
        self.clock = clock
        self.queue: deque = deque()
        self.running: list = []
        self.done: list = []
        self.in_use = 0
        self.peak_in_use = 0
        self.rounds = 0
        self.max_members = 0
        self.feed: Optional[Callable[[], None]] = None  # submits jobs that arrived meanwhile

    def submit(self, job: Job):
        job.est_bytes = int(self.be.estimate(job))
        if job.est_bytes > self.budget:
            raise ValueError(f"job {job.job_id} needs {job.est_bytes} B, above the whole budget")
        self.queue.append(job)

    def _admit(self):
        """Creates systems for queued jobs in arrival order while they fit."""
        admitted = []
        while self.queue and self.in_use + self.queue[0].est_bytes <= self.budget:
            job = self.queue.popleft()
            job.handle = self.be.create(job)
            job.admitted = self.clock()
            self.in_use += job.est_bytes
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            admitted.append(job)
        return admitted

    def _retire(self, job: Job):
        job.result = self.be.finish(job.handle)
        self.be.close(job.handle)
        job.handle = None
        job.finished = self.clock()
        self.in_use -= job.est_bytes
        self.done.append(job)

    def step(self) -> bool:
        """One round: admit, launch a round of the batch, then (while the GPU
        works) admit more, wait, and retire finished jobs.  Returns False when
        there is nothing to run."""
        if self.feed:
            self.feed()
        for job in self._admit():
            self._join(job)
        if not self.running:
            return False
        left = min(j.nsteps - j.steps_done for j in self.running)
        k = min(self.round_steps, (left // self.theta) * self.theta)
        if k > 0:
            self.be.run(k)
            for j in self.running:
                j.steps_done += k
        self.rounds += 1
        if self.feed:
            self.feed()
        late = self._admit()  # overlaps the round on the GPU (uploads, binning)
        self.be.sync()
        for j in list(self.running):
            rem = j.nsteps - j.steps_done
            if rem < self.theta:
                self.be.remove(j.handle)
                self.running.remove(j)
                if rem:
                    self.be.run_alone(j.handle, rem)
                    j.steps_done += rem
                self._retire(j)
        for job in late:
            self._join(job)
        return True

    def _join(self, job: Job):
        if job.nsteps < self.theta:  # too short to share a round: run alone
            if job.nsteps:
                self.be.run_alone(job.handle, job.nsteps)
                job.steps_done = job.nsteps
            self._retire(job)
            return
        self.be.add(job.handle)
        self.running.append(job)
        self.max_members = max(self.max_members, len(self.running))

    def idle(self) -> bool:
        return not self.queue and not self.running


def serve_trace(server: Server, jobs: list, clock: Callable[[], float] = time.perf_counter,
                sleep: Callable[[float], None] = time.sleep) -> dict:
    """Replays an arrival trace (job.arrival in seconds from the start) in
    real time through `server`; returns latency percentiles and throughput."""
    pending = deque(sorted(jobs, key=lambda j: j.arrival))
    t0 = clock()
    for j in pending:
        j.arrival += t0

    def feed():
        now = clock()
        while pending and pending[0].arrival <= now:
            server.submit(pending.popleft())

    server.feed = feed
    while pending or not server.idle():
        if not server.step():
            if pending:
                sleep(max(0.0, min(pending[0].arrival - clock(), 0.05)))
    wall = clock() - t0
    return summarize(server.done, wall)


def serve_serial(backend, jobs: list, clock: Callable[[], float] = time.perf_counter,
                 sleep: Callable[[float], None] = time.sleep) -> dict:
    """The same trace one job at a time: each job is created, run alone to
    completion and read back before the next (FIFO) starts."""
    pending = deque(sorted(jobs, key=lambda j: j.arrival))
    t0 = clock()
    for j in pending:
        j.arrival += t0
    done = []
    while pending:
        j = pending.popleft()
        wait = j.arrival - clock()
        if wait > 0:
            sleep(wait)
        h = backend.create(j)
        j.admitted = clock()
        backend.run_alone(h, j.nsteps)
        j.steps_done = j.nsteps
        j.result = backend.finish(h)
        backend.close(h)
        j.finished = clock()
        done.append(j)
    wall = clock() - t0
    return summarize(done, wall)


def summarize(done: list, wall: float) -> dict:
    lat = np.array([j.latency for j in done]) if done else np.zeros(1)
    replica_steps = sum(j.nsteps for j in done)
    particle_steps = sum(j.nsteps * j.n for j in done)
    return {"jobs": len(done), "wall_s": wall,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()),
            "replica_steps_per_s": replica_steps / wall if wall > 0 else 0.0,
            "particle_steps_per_s": particle_steps / wall if wall > 0 else 0.0}
