"""Serving loop: polymerisation jobs of different sizes arrive over time and
share one GPU through one prx_batch (continuous batching).

Each job is a system (positions, velocities, types, states, a reaction
scheme, a seed) and a number of MD steps.  The loop:

  * admits queued jobs while a slot and device memory are free
    (prx_estimate_bytes against the batch's budget; prx_batch_admit refuses
    with PRX_ENOMEM otherwise).  Jobs are taken in arrival order, but a job
    that does not fit lets later jobs that fit go ahead (backfilling) until it
    has waited `patience` seconds; then it holds the queue until it fits.  An
    admitted job's system is created (uploaded and binned) while the batch is
    busy on the GPU;
  * queues epochs of the batch (prx_batch_step_epoch: whole reaction
    intervals, never past a job's step count; a job with less than an
    interval left finishes alone on its own stream), with no host wait while
    at most two epochs are queued;
  * retires the jobs that prx_batch_poll reports finished: their bonds and
    states are read back, their memory freed, and their latency (arrival to
    result) recorded.

A job's result does not depend on which other jobs shared the GPU with it
(the batch runs each member's own kernels on its own data).  All simulation
work runs in the library's CUDA kernels and the admission, epoch and
completion bookkeeping in its C runtime; this module only decides which job
to admit next.  The backend interface is small so that the scheduling logic
can be tested without a GPU.
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
    handle: Any = None
    slot: int = -1

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival


class PolyrxBackend:
    """Backend on the polyrx C ABI: prx_create, prx_batch_admit,
    prx_batch_step_epoch, prx_batch_poll."""

    def __init__(self, P, stream=None, positions: bool = False, mem_budget: int = 0,
                 max_slots: int = 0):
        self.P = P
        self.batch = P.Batch(stream=stream, max_slots=max_slots, mem_budget=mem_budget)
        self.positions = positions

    def estimate(self, job: Job) -> int:
        return self.P.prx_estimate_bytes(job.system["desc"], job.system.get("reaction"))

    def fits(self, nbytes: int) -> bool:
        st = self.batch.stats()
        if st["max_slots"] and st["slots_used"] >= st["max_slots"]:
            return False
        return not st["mem_budget"] or st["bytes_admitted"] + nbytes <= st["mem_budget"]

    def create(self, job: Job):
        s = job.system
        g = self.P.System(s["desc"], s["pos"], s.get("vel"), s["type"], s["state"])
        if s.get("reaction") is not None:
            g.set_reaction(s["reaction"])
        return g

    def admit(self, h, nsteps: int):
        """The job's slot, or None when the batch refused it (no slot or memory)."""
        return self.batch.admit(h, nsteps)

    def epoch(self, max_steps: int) -> int:
        return self.batch.step_epoch(max_steps)

    def poll(self) -> list:
        return self.batch.poll()

    def run_alone(self, h, nsteps: int):
        h.run(nsteps)

    def finish(self, h):
        """Reads the job's result back (synchronises its own stream)."""
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

    mem_budget : device bytes the admitted jobs may occupy together (the
                 backend's batch enforces it; the server only uses it to
                 refuse jobs that could never fit)
    round_steps: most MD steps per epoch (a multiple of theta)
    theta      : the reaction interval shared by the jobs
    patience   : seconds a job that does not fit lets later jobs go ahead
    clock      : time source (seconds)
    """

    def __init__(self, backend, mem_budget: int, round_steps: int = 200, theta: int = 10,
                 clock: Callable[[], float] = time.perf_counter, patience: float = 0.5,
                 idle_wait: Callable[[], None] = lambda: time.sleep(2e-4)):
        if round_steps % theta:
            raise ValueError("round_steps must be a multiple of theta")
        self.be = backend
        self.budget = int(mem_budget)
        self.round_steps = round_steps
        self.theta = theta
        self.clock = clock
        self.patience = patience
        self.idle_wait = idle_wait
        self.queue: deque = deque()
        self.by_slot: dict = {}
        self.done: list = []
        self.in_use = 0
        self.peak_in_use = 0
        self.rounds = 0
        self.max_members = 0
        self._resident_sum = 0
        self.feed: Optional[Callable[[], None]] = None  # submits jobs that arrived meanwhile

    def submit(self, job: Job):
        job.est_bytes = int(self.be.estimate(job))
        if job.est_bytes > self.budget:
            raise ValueError(f"job {job.job_id} needs {job.est_bytes} B, above the whole budget")
        self.queue.append(job)

    def _admit(self):
        """Creates and admits queued jobs that fit, in arrival order with
        backfilling past a job that does not fit (until it ran out of
        patience)."""
        now = self.clock()
        for job in list(self.queue):
            if not self.be.fits(job.est_bytes):
                if now - job.arrival > self.patience:
                    break  # this job holds the queue until it fits
                continue
            h = self.be.create(job)
            slot = self.be.admit(h, job.nsteps)
            if slot is None:  # refused after all: try again later
                self.be.close(h)
                continue
            self.queue.remove(job)
            job.handle, job.slot, job.admitted = h, slot, self.clock()
            self.by_slot[slot] = job
            self.in_use += job.est_bytes
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            self.max_members = max(self.max_members, len(self.by_slot))

    def _retire(self, job: Job):
        job.result = self.be.finish(job.handle)
        job.finished = self.clock()
        self.be.close(job.handle)
        job.handle = None
        self.in_use -= job.est_bytes
        self.done.append(job)

    def step(self) -> bool:
        """One round: admit, queue an epoch, admit jobs that arrived
        meanwhile (their creation overlaps the epoch on the GPU), retire the
        finished ones.  Returns False when there is nothing to run."""
        if self.feed:
            self.feed()
        self._admit()
        if not self.by_slot:
            return False
        k = self.be.epoch(self.round_steps)
        self.rounds += 1
        self._resident_sum += len(self.by_slot)
        if self.feed:
            self.feed()
        self._admit()
        finished = self.be.poll()
        for slot in finished:
            self._retire(self.by_slot.pop(slot))
        if k == 0 and not finished:
            self.idle_wait()  # only jobs finishing alone are left: let them run
        return True

    def mean_members(self) -> float:
        return self._resident_sum / self.rounds if self.rounds else 0.0

    def idle(self) -> bool:
        return not self.queue and not self.by_slot


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
        j.result = backend.finish(h)
        j.finished = clock()
        backend.close(h)
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
