"""Continuous-batching serving loop for IsoMP simulation jobs.

Jobs (N, number of steps, h, precision, initial state) arrive over time.  Jobs
of like N and precision form a class; each class has its own first-come,
first-served queue.  The head of a class's queue is admitted when its plan's
device footprint fits the memory budget and the class's step latency allows
it: a class with no resident job always takes its head job; otherwise a new job
joins only after the class has completed a step with its current set and while
the class's measured step latency (moving average) is below the target.  Under
overload the queues absorb the excess (reported as queueing delay) instead of
the batches growing until every resident job's step takes seconds.  An admitted
job's state stays resident on the device until its last step.  Each class is
advanced by its own worker thread on its own CUDA stream (smaller N at higher
priority), one batched step (grouped kernels over all the class's jobs) per
iteration.  Jobs that are admitted while others are running join their class's
batch at its next step, and classes run concurrently on the device.  A class's
batch is rebuilt only when its resident set changes.  All arithmetic runs in
the library's kernels; this module only schedules.

Reported: per-step latency of resident jobs (time between a job's consecutive
completed steps; p50/p99, overall and per class), aggregate job-steps/s,
queueing delay (arrival to admission) and the peak of admitted footprint.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
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
    last_done: float


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs) * 1e3, q)) if len(xs) else None


def next_admission(queues, resident, used, budget, stepped, ema, target, estimate):
    """The class whose head job is admitted next, or None (the admission policy).

    queues: class -> deque of waiting jobs (FIFO per class); classes are tried in
    the order of their head job's arrival.  resident: class -> number of resident
    jobs.  A head job fits when its plan footprint estimate(N, precision) fits the
    remaining budget, or nothing at all is resident.  A class with resident jobs
    admits another only after a completed step with its current set (stepped)
    and while its step-time average ema[class] is below target (seconds; None:
    footprint only).
    """
    anything = sum(resident.values()) > 0
    for cls in sorted((c for c in queues if queues[c]), key=lambda c: queues[c][0].arrival):
        head = queues[cls][0]
        if used + estimate(head.N, head.precision) > budget and anything:
            continue
        if resident.get(cls) and target is not None and not (stepped.get(cls) and ema.get(cls, 0.0) < target):
            continue
        return cls
    return None


class Server:
    def __init__(self, budget_bytes: int, tol: float = 1e-12, maxit: int = 50, graph: bool = False,
                 target_step_ms: float | None = 100.0):
        """target_step_ms: step latency above which a class admits no further job
        (None: admission by memory footprint alone)."""
        self.budget = int(budget_bytes)
        self.tol = tol
        self.maxit = maxit
        self.graph = graph
        self.target = None if target_step_ms is None else float(target_step_ms) * 1e-3

    def run(self, jobs, time_limit: float | None = None, keep_results: bool = False, clock=time.perf_counter):
        """Serve `jobs`; returns a report dict (results by job id if keep_results)."""
        import torch

        dev = torch.cuda.current_device()
        low, high = torch.cuda.Stream.priority_range()   # e.g. (0, -5): lower number = higher priority
        # admissions copy state on the highest-priority stream, never waiting on running steps
        upload = torch.cuda.Stream(priority=high)
        sizes = sorted({j.N for j in jobs})

        def class_priority(N):   # smaller matrices are the latency-sensitive classes
            rank = sizes.index(N)
            span = max(1, len(sizes) - 1)
            return int(round(high + (low - high) * rank / span))
        lock = threading.Lock()
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        queues: dict[tuple, collections.deque] = collections.defaultdict(collections.deque)
        ema: dict[tuple, float] = {}            # moving average of the class's step time (s)
        stepped: dict[tuple, bool] = {}         # a step completed since the class's last admission
        classes: dict[tuple, dict[int, _Resident]] = {}
        dirty: dict[tuple, bool] = {}
        workers: dict[tuple, threading.Thread] = {}
        lat: dict[tuple, list] = collections.defaultdict(list)
        max_res: dict[tuple, int] = collections.defaultdict(int)   # peak resident jobs per class
        qdelay, results, errors, admit_times = [], {}, [], []
        pinned = {}
        st = {"used": 0, "peak": 0, "steps": 0, "completed": 0, "batched": 0, "stop": False}
        t0 = clock()

        def worker(cls):
            torch.cuda.set_device(dev)
            stream = torch.cuda.Stream(priority=class_priority(cls[0]))
            batch, order = None, []
            try:
                while True:
                    with lock:
                        res = dict(classes[cls])
                        changed = dirty[cls]
                        dirty[cls] = False
                        stop = st["stop"]
                    if stop:   # time limit: leave; resident jobs are released by the caller
                        if batch is not None:
                            batch.close()
                        return
                    if not res:
                        if batch is not None:
                            batch.close()
                            batch = None
                        if not pending and not queues[cls]:
                            with lock:
                                if not classes[cls] and not pending and not queues[cls]:
                                    return
                        time.sleep(0.001)
                        continue
                    if changed or batch is None:
                        if batch is not None:
                            batch.close()
                        order = sorted(res)
                        batch = z.Batch([res[j].plan for j in order], [res[j].W for j in order],
                                        [res[j].job.h for j in order])
                        if self.graph:
                            batch.set_graph(True)
                    t_start = clock() - t0
                    with torch.cuda.stream(stream):
                        batch.step(self.tol, self.maxit, stream=stream, allow_not_converged=True)
                    t_done = clock() - t0
                    finished = []
                    with lock:
                        st["batched"] += 1
                        dt = t_done - t_start
                        ema[cls] = dt if cls not in ema else 0.7 * ema[cls] + 0.3 * dt
                        stepped[cls] = True
                        for j in order:
                            r = classes[cls][j]
                            lat[cls].append(t_done - r.last_done)
                            r.last_done = t_done
                            r.remaining -= 1
                            st["steps"] += 1
                            if r.remaining == 0:
                                finished.append(r)
                    if finished:
                        batch.close()
                        batch = None
                        for r in finished:
                            if keep_results:
                                results[r.job.jid] = r.W.cpu().numpy()
                            r.plan.close()
                        with lock:
                            for r in finished:
                                del classes[cls][r.job.jid]
                                st["used"] -= r.bytes
                                st["completed"] += 1
                            dirty[cls] = True
            except Exception as e:   # surfaced to the caller after the run
                errors.append(repr(e))
                with lock:
                    st["stop"] = True

        while True:
            now = clock() - t0
            if time_limit is not None and now > time_limit or errors:
                with lock:
                    st["stop"] = True
                break
            with lock:
                while pending and pending[0].arrival <= now:
                    j = pending.popleft()
                    queues[(j.N, j.precision)].append(j)
            admitted = False
            while True:   # per class first come, first served; classes by their head's arrival
                if time_limit is not None and clock() - t0 > time_limit:
                    break
                job = None
                with lock:
                    cls = next_admission(queues, {c: len(v) for c, v in classes.items()}, st["used"], self.budget,
                                         stepped, ema, self.target, z.plan_estimate_bytes)
                    if cls is not None:
                        job = queues[cls].popleft()
                        stepped[cls] = False
                if job is None:
                    break
                need = z.plan_estimate_bytes(job.N, job.precision)
                ta = clock()
                plan = z.Plan(job.N, job.precision)
                tb = clock()
                src = pinned.get(id(job.W0))   # initial states shared by jobs are pinned once
                if src is None:
                    src = torch.from_numpy(np.ascontiguousarray(job.W0)).pin_memory()
                    pinned[id(job.W0)] = src
                with torch.cuda.stream(upload):
                    W = src.to("cuda", non_blocking=True)
                upload.synchronize()
                admit_times.append((tb - ta, clock() - tb))
                t_adm = clock() - t0
                cls = (job.N, job.precision)
                with lock:
                    classes.setdefault(cls, {})[job.jid] = _Resident(job, plan, W, need, job.nsteps, t_adm)
                    max_res[cls] = max(max_res[cls], len(classes[cls]))
                    dirty[cls] = True
                    st["used"] += need
                    st["peak"] = max(st["peak"], st["used"])
                    qdelay.append(t_adm - job.arrival)
                    if cls not in workers or not workers[cls].is_alive():
                        th = threading.Thread(target=worker, args=(cls,), daemon=True)
                        workers[cls] = th
                        th.start()
                admitted = True
            with lock:
                empty = not pending and not any(queues.values()) and not any(classes.values())
            if empty:
                break
            if not admitted:
                time.sleep(0.001)
        for th in list(workers.values()):
            th.join()
        wall = clock() - t0
        for c in classes.values():
            for r in c.values():
                r.plan.close()
        if errors:
            raise RuntimeError("serving worker failed: " + errors[0])
        allat = [x for v in lat.values() for x in v]
        return {
            "wall_s": wall,
            "job_steps": st["steps"],
            "job_steps_per_s": st["steps"] / wall if wall > 0 else 0.0,
            "batched_steps": st["batched"],
            "jobs_completed": st["completed"],
            "jobs_admitted": len(qdelay),
            "jobs_left_queued": sum(len(q) for q in queues.values()) + len(pending),
            "target_step_ms": None if self.target is None else self.target * 1e3,
            "step_latency_ms_p50": _pct(allat, 50),
            "step_latency_ms_p99": _pct(allat, 99),
            "per_class": {f"N={k[0]},{'split' if k[1] == z.PRECISION_SPLIT else 'fp64'}":
                          {"job_steps": len(v), "p50_ms": _pct(v, 50), "p99_ms": _pct(v, 99),
                           "max_resident": max_res[k]}
                          for k, v in lat.items()},
            "queue_delay_s_p50": float(np.percentile(qdelay, 50)) if qdelay else None,
            "peak_admitted_bytes": st["peak"],
            "admit_plan_ms_mean": float(np.mean([a for a, _ in admit_times]) * 1e3) if admit_times else None,
            "admit_upload_ms_mean": float(np.mean([b for _, b in admit_times]) * 1e3) if admit_times else None,
            "results": results,
        }
