"""Continuous-batching serving loop for IsoMP simulation jobs.

Jobs (N, number of steps, h, precision, initial state) arrive over time.  A job
is admitted when its plan's device footprint fits the memory budget (first
come, first served); its state then stays resident on the device until its
last step.  Every loop iteration advances all resident jobs by one IsoMP step
in one batched step (grouped kernels over jobs of any mix of N), so jobs that
arrive while others are running join the next step -- their work overlaps on
the device with the jobs already resident.  The batch is rebuilt only when the
resident set changes.  All arithmetic runs in the library's kernels; this
module only schedules.

Reported: per-step latency of resident jobs (time between a job's consecutive
completed steps; p50/p99), aggregate job-steps/s, queueing delay (arrival to
admission), and the peak of admitted footprint.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import zeitlin as z


@dataclasses.dataclass
class Job:
    jid: int
    N: int
    nsteps: int
    h: float
    precision: int
    arrival: float          # seconds after the start of the run
    W0: np.ndarray          # complex128 initial vorticity matrix (host)


@dataclasses.dataclass
class _Resident:
    job: Job
    plan: z.Plan
    W: object               # device tensor
    bytes: int
    remaining: int
    admitted: float
    last_done: float


class Server:
    def __init__(self, budget_bytes: int, tol: float = 1e-12, maxit: int = 50, graph: bool = False):
        self.budget = int(budget_bytes)
        self.tol = tol
        self.maxit = maxit
        self.graph = graph

    def run(self, jobs, time_limit: float | None = None, keep_results: bool = False, clock=time.perf_counter):
        """Serve `jobs` (sorted or not by arrival).  Returns a report dict."""
        import torch

        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        queue = collections.deque()
        active: dict[int, _Resident] = {}
        used = peak = 0
        batch, dirty = None, True
        lat, qdelay, results = [], [], {}
        steps_done = 0
        completed = 0
        batched_steps = 0
        t0 = clock()
        while pending or queue or active:
            now = clock() - t0
            if time_limit is not None and now > time_limit:
                break
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            while queue:   # first come, first served, by device footprint
                job = queue[0]
                need = z.plan_estimate_bytes(job.N, job.precision)
                if used + need > self.budget and active:
                    break
                queue.popleft()
                plan = z.Plan(job.N, job.precision)
                W = torch.from_numpy(np.ascontiguousarray(job.W0)).cuda()
                t_adm = clock() - t0
                active[job.jid] = _Resident(job, plan, W, need, job.nsteps, t_adm, t_adm)
                qdelay.append(t_adm - job.arrival)
                used += need
                peak = max(peak, used)
                dirty = True
            if not active:
                if pending:   # idle until the next arrival
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - (clock() - t0))))
                continue
            if dirty:
                if batch is not None:
                    batch.close()
                res = list(active.values())
                batch = z.Batch([r.plan for r in res], [r.W for r in res], [r.job.h for r in res])
                if self.graph:
                    batch.set_graph(True)
                order = [r.job.jid for r in res]
                dirty = False
            rc, st = batch.step(self.tol, self.maxit, allow_not_converged=True)
            t_done = clock() - t0
            batched_steps += 1
            for jid in order:
                r = active[jid]
                lat.append(t_done - r.last_done)
                r.last_done = t_done
                r.remaining -= 1
                steps_done += 1
            for jid in list(order):
                r = active[jid]
                if r.remaining == 0:
                    if keep_results:
                        results[jid] = r.W.cpu().numpy()
                    used -= r.bytes
                    r.plan.close()
                    del active[jid]
                    completed += 1
                    dirty = True
            if dirty and batch is not None:
                batch.close()
                batch = None
        wall = clock() - t0
        if batch is not None:
            batch.close()
        for r in active.values():
            r.plan.close()
        lat_ms = np.asarray(lat) * 1e3
        return {
            "wall_s": wall,
            "job_steps": steps_done,
            "job_steps_per_s": steps_done / wall if wall > 0 else 0.0,
            "batched_steps": batched_steps,
            "jobs_completed": completed,
            "jobs_admitted": len(qdelay),
            "jobs_left_queued": len(queue) + len(pending),
            "step_latency_ms_p50": float(np.percentile(lat_ms, 50)) if len(lat_ms) else None,
            "step_latency_ms_p99": float(np.percentile(lat_ms, 99)) if len(lat_ms) else None,
            "queue_delay_s_p50": float(np.percentile(qdelay, 50)) if qdelay else None,
            "peak_admitted_bytes": peak,
            "results": results,
        }
