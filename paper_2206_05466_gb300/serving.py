"""Continuous-batching serving loop for IsoMP simulation jobs.

Jobs (N, number of steps, h, precision, initial state) arrive over time.  Jobs
of like N and precision form a class; each class has its own first-come,
first-served queue.  Before serving, each class's solo step time (a batched
step of one and of two instances alone on the device) is calibrated.  The head
of a class's queue is admitted when its plan's device footprint fits the memory
budget and the admission policy (next_admission) allows it: by default one
class is resident at a time (measured: two classes sharing the device, even of
comparable step time, put the lighter one's p99 step latency at 5-8 times its
solo step time; a setting allows more, and then only classes whose solo step
times are within a factor 8 share the device), and a
resident class takes another job only after it completed a step with its
current set, while its measured step time stays below 0.8 x 2 times its solo
step time with one job (a batch's step time grows with its size; past a few
dozen small jobs the device is full and larger batches only add latency) and
its solo step time with one more job stays below an absolute target; after
a session of 20 s a class stops taking jobs while other classes wait, so that
the resident classes rotate.  Under overload the queues absorb the excess
(reported as queueing delay).  An admitted job's state stays resident on the
device until its last step.  Each class is advanced by its own worker thread on
its own CUDA stream, one batched step (grouped kernels over all the class's
jobs) per iteration; jobs admitted while others run join their class's batch
at its next step (when several classes are allowed, they run concurrently).
A class's batch is rebuilt only when its resident set changes, and the new
batch is built on a helper thread while the current one keeps stepping: the
worker swaps it in between two steps, so a rebuild does not pause the class.
All arithmetic runs in the library's kernels; this module only schedules.

Reported: per-step latency of resident jobs (time between a job's consecutive
completed steps; p50/p99, overall and per class), aggregate job-steps/s,
queueing delay (arrival to admission) and the peak of admitted footprint.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import gc
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
    done: bool = False      # all steps taken; stepped along (results ignored) until the next rebuild


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs) * 1e3, q)) if len(xs) else None


def _step_breakdown(step_log):
    """Batched-step times per class and tag: count, p50 and p99 (ms)."""
    out = {}
    for cls in sorted({c for c, _, _ in step_log}):
        name = f"N={cls[0]},{'split' if cls[1] == z.PRECISION_SPLIT else 'fp64'}"
        rows = [(dt, tags) for c, dt, tags in step_log if c == cls]
        groups = {"all": [dt for dt, _ in rows], "untagged": [dt for dt, t in rows if not t]}
        for tag in ("swap", "admission", "more_sweeps", "gc", "building"):
            groups[tag] = [dt for dt, t in rows if tag in t]
        out[name] = {k: {"n": len(v), "p50": _pct(v, 50), "p99": _pct(v, 99)} for k, v in groups.items() if v}
    return out


def solo_step_s(solo, cls, n):
    """Calibrated step time of class `cls` with n resident jobs, running alone on the
    device: solo[cls] = (t1, per_job), t1 + per_job * (n - 1) seconds."""
    t1, per = solo[cls]
    return t1 + per * max(0, n - 1)


def next_admission(queues, resident, used, budget, stepped, ema, solo, estimate, factor=2.0, headroom=0.8,
                   max_active=2, target=None, active_since=None, now=0.0, session_s=None, compat=None):
    """The class whose head job is admitted next, or None (the admission policy).

    queues: class -> deque of waiting jobs (FIFO per class); classes are tried in
    the order of their head job's arrival.  resident: class -> number of resident
    jobs; a class with resident jobs is active.
      * Device sharing: at most `max_active` classes are active at once, so that a
        class's steps share the device with at most max_active - 1 others (with
        two, each gets at least about half the device: step time <= 2x solo).
      * Memory: the head job's plan footprint estimate(N, precision) must fit the
        remaining budget, unless nothing at all is resident.
      * Latency: an active class admits another job only after it completed a step
        with its current set (stepped), while its measured step time ema[cls], and its
        calibrated solo step time with one more job, stay below `headroom` x `factor`
        times its solo step time with one job (the headroom leaves room for the jobs
        of the next admission burst, so that the class's steps stay within `factor`
        times that solo time), and while the
        calibrated solo step time with one more job stays within the absolute
        `target` (seconds).  (Measured: a batch's step time grows with its size, and
        past a few dozen small jobs the device is full, so larger batches only add
        latency.)  With neither (both None) admission is by footprint and the number
        of active classes alone.
      * Sessions: an active class that has been active for more than session_s
        seconds (active_since[cls]) admits no further job while a class that is not
        active has jobs waiting, so that the active classes drain and free their
        place (None: no limit).
      * Compatibility: a class becomes active next to others only if its solo step
        time with one job and theirs are within a factor `compat` of each other
        (None: any), so that millisecond steps never share the device with
        kernels whose CTAs hold an SM for longer than such a step.
    """
    active = {c for c, n in resident.items() if n > 0}
    anything = bool(active)
    waiting_inactive = any(queues[c] for c in queues if c not in active)
    for cls in sorted((c for c in queues if queues[c]), key=lambda c: queues[c][0].arrival):
        head = queues[cls][0]
        if used + estimate(head.N, head.precision) > budget and anything:
            continue
        n = resident.get(cls, 0)
        if n == 0:
            if len(active) >= max_active:
                continue
            if compat is not None and any(max(solo[cls][0], solo[a][0]) > compat * min(solo[cls][0], solo[a][0])
                                          for a in active):
                continue
            return cls
        if factor is not None or target is not None:
            if not stepped.get(cls):
                continue
            gate = None if factor is None else headroom * factor * solo_step_s(solo, cls, 1)
            if factor is not None and (cls not in ema or ema[cls] > gate):
                continue
            if factor is not None and solo_step_s(solo, cls, n + 1) > gate:   # the calibrated cost of one more
                continue
            if target is not None and solo_step_s(solo, cls, n + 1) > target:
                continue
        if (session_s is not None and active_since is not None and waiting_inactive
                and now - active_since.get(cls, now) > session_s):
            continue
        return cls
    return None


class Server:
    def __init__(self, budget_bytes: int, tol: float = 1e-12, maxit: int = 50, graph: bool = False,
                 target_step_ms: float | None = 100.0, latency_factor: float = 2.0, max_active: int = 1,
                 session_s: float | None = 20.0, compat: float | None = 8.0, burst: int = 4):
        """target_step_ms: a class admits another job only while its solo step time with
        that job stays below this (None: no absolute bound); latency_factor: ... and
        while its measured step time is within this factor of its solo step time;
        max_active: classes resident at once; session_s: after this long, an active
        class stops admitting while other classes wait (None: no limit); compat:
        largest ratio of solo step times of two classes resident together (None:
        any); burst: jobs a resident class may take after one completed step (one
        batch rebuild for all of them)."""
        self.budget = int(budget_bytes)
        self.tol = tol
        self.maxit = maxit
        self.graph = graph
        self.target = None if target_step_ms is None else float(target_step_ms) * 1e-3
        self.factor = None if latency_factor is None else float(latency_factor)
        self.max_active = int(max_active)
        self.session_s = session_s
        self.compat = compat
        self.burst = max(1, int(burst))
        self.headroom = 0.8
        self.step_series = None   # a list here receives (class, start s, seconds, jobs, sweeps, tags) per step

    def calibrate(self, classes, W0s, h=0.01, reps=2):
        """Solo step time of each class (N, precision), alone on the device: batched steps
        of one and of two instances (seconds), as {cls: (t1, per_job)}."""
        import torch

        out = {}
        for cls in classes:
            N, prec = cls
            times = []
            for n in (1, 2):
                plans = [z.Plan(N, prec) for _ in range(n)]
                Ws = [torch.from_numpy(np.ascontiguousarray(W0s[cls])).cuda() for _ in range(n)]
                b = z.Batch(plans, Ws, [h] * n)
                b.step(self.tol, self.maxit, allow_not_converged=True)   # warm-up
                torch.cuda.synchronize()
                t = time.perf_counter()
                for _ in range(reps):
                    b.step(self.tol, self.maxit, allow_not_converged=True)
                torch.cuda.synchronize()
                times.append((time.perf_counter() - t) / reps)
                b.close()
                for p in plans:
                    p.close()
            out[cls] = (times[0], max(0.0, times[1] - times[0]))
        return out

    def run(self, jobs, time_limit: float | None = None, keep_results: bool = False, clock=time.perf_counter,
            solo=None):
        """Serve `jobs`; returns a report dict (results by job id if keep_results).
        solo: calibrated solo step times ({cls: (t1, per_job)}); measured with
        calibrate() on the jobs' classes when None."""
        import torch

        if solo is None:
            firsts = {}
            for j in jobs:
                firsts.setdefault((j.N, j.precision), j.W0)
            tc = time.perf_counter()
            solo = self.calibrate(sorted(firsts), firsts)
            calib_s = time.perf_counter() - tc
        else:
            calib_s = 0.0

        dev = torch.cuda.current_device()
        low, high = torch.cuda.Stream.priority_range()   # e.g. (0, -5): lower number = higher priority
        # admissions copy state on the highest-priority stream, never waiting on running steps
        upload = torch.cuda.Stream(priority=high)

        def class_priority(N):   # the two active classes share the device evenly
            return low
        lock = threading.Lock()
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        pending_arrivals = pending   # (the workers' name for it)
        queues: dict[tuple, collections.deque] = collections.defaultdict(collections.deque)
        ema: dict[tuple, float] = {}            # moving average of the class's step time (s)
        active_since: dict[tuple, float] = {}   # start of the class's current session (s)
        res_hist: dict[tuple, list] = collections.defaultdict(list)   # resident count at each step
        stepped: dict[tuple, bool] = {}         # a step completed since the class's last admission
        took: dict[tuple, int] = collections.defaultdict(int)   # jobs admitted since the class's last step
        classes: dict[tuple, dict[int, _Resident]] = {}
        dirty: dict[tuple, bool] = {}
        workers: dict[tuple, threading.Thread] = {}
        lat: dict[tuple, list] = collections.defaultdict(list)
        max_res: dict[tuple, int] = collections.defaultdict(int)   # peak resident jobs per class
        qdelay, results, errors, admit_times = [], {}, [], []
        # per batched step: (class, seconds, tags) -- tags: the first step after a batch swap,
        # an admission (plan creation and upload) overlapping the step, more sweeps than the
        # class's previous step (a second convergence check inside the step)
        step_log = []
        admitting = [0]
        gc_runs = [0]   # garbage collections started so far (any thread)

        def _gc_cb(phase, info):
            if phase == "start":
                gc_runs[0] += 1
        gc.callbacks.append(_gc_cb)
        pinned = {}
        st = {"used": 0, "peak": 0, "steps": 0, "completed": 0, "batched": 0, "stop": False}
        t0 = clock()

        def worker(cls):
            torch.cuda.set_device(dev)
            stream = torch.cuda.Stream(priority=class_priority(cls[0]))
            builder = concurrent.futures.ThreadPoolExecutor(max_workers=1)
            batch, order = None, []
            pending = None       # (order, future of the batch being built for that order)
            prev_max = 0         # most sweeps any job took in the previous step
            want = False         # the resident set changed since the last build was started
            since = 0   # batched steps since the last rebuild

            def build(ord_, res_):
                torch.cuda.set_device(dev)
                b = z.Batch([res_[j].plan for j in ord_], [res_[j].W for j in ord_], [res_[j].job.h for j in ord_])
                if self.graph:
                    b.set_graph(True)
                return b

            def swap_in(new_order, new_batch):
                # the old batch is idle (its last step synchronised); its finished jobs
                # that the new batch leaves out are released now
                nonlocal batch, order, since
                if batch is not None:
                    batch.close()
                keep = set(new_order)
                with lock:
                    gone = [r for j, r in classes[cls].items() if j not in keep and r.done]
                    for r in gone:
                        del classes[cls][r.job.jid]
                        st["used"] -= r.bytes
                for r in gone:
                    r.plan.close()
                batch, order, since = new_batch, new_order, 0

            try:
                while True:
                    with lock:
                        res = dict(classes[cls])
                        if dirty[cls]:
                            want = True
                        dirty[cls] = False
                        stop = st["stop"]
                    if stop:   # time limit: leave; resident jobs are released by the caller
                        if pending is not None:
                            pb = pending[1].result()
                            pb.close()
                        if batch is not None:
                            batch.close()
                        builder.shutdown()
                        return
                    live = {j: r for j, r in res.items() if not r.done}
                    if pending is not None and pending[1].done():
                        new_order, fut = pending
                        pending = None
                        swap_in(new_order, fut.result())
                        continue
                    if not live:
                        # nothing left to step: release everything at once
                        if pending is not None:
                            pending[1].result().close()
                            pending = None
                        if batch is not None or res:
                            swap_in([], None)
                        want = False
                        if not pending_jobs(cls):
                            with lock:
                                if not classes[cls] and not pending_jobs(cls):
                                    builder.shutdown()
                                    return
                        time.sleep(0.001)
                        continue
                    # Finished jobs leave the batch at the next rebuild: together with the next
                    # admission, once a quarter of the batch has finished, or after 32 steps.
                    nz = sum(1 for j in order if res.get(j) is not None and res[j].done)
                    if nz and (nz * 4 >= len(order) or since >= 32):
                        want = True
                    if want and pending is None:
                        new_order = sorted(live)
                        want = False
                        if batch is None:   # nothing to step meanwhile: build here
                            swap_in(new_order, build(new_order, res))
                        else:
                            pending = (new_order, builder.submit(build, new_order, res))
                    t_start = clock() - t0
                    adm0, gc0, bld0 = admitting[0], gc_runs[0], pending is not None
                    with torch.cuda.stream(stream):
                        _, sts = batch.step(self.tol, self.maxit, stream=stream, allow_not_converged=True)
                    t_done = clock() - t0
                    mx = max(x["iters"] for x in sts)
                    tags = (("swap",) if since == 0 else ()) + (("admission",) if adm0 or admitting[0] else ()) + \
                        (("more_sweeps",) if prev_max and mx > prev_max else ()) + \
                        (("gc",) if gc_runs[0] != gc0 else ()) + (("building",) if bld0 else ())
                    prev_max = mx
                    step_log.append((cls, t_done - t_start, tags))
                    if self.step_series is not None:
                        self.step_series.append((cls, t_start, t_done - t_start, len(order), mx, tags))
                    since += 1
                    finished = []
                    with lock:
                        st["batched"] += 1
                        dt = t_done - t_start
                        ema[cls] = dt if cls not in ema else 0.7 * ema[cls] + 0.3 * dt
                        stepped[cls] = True
                        took[cls] = 0
                        res_hist[cls].append(len(order))
                        for j in order:
                            r = classes[cls][j]
                            if r.done:
                                continue
                            lat[cls].append(t_done - r.last_done)
                            r.last_done = t_done
                            r.remaining -= 1
                            st["steps"] += 1
                            if r.remaining == 0:
                                r.done = True
                                finished.append(r)
                                st["completed"] += 1
                    for r in finished:   # the state after the job's last step (the step has synchronised)
                        if keep_results:
                            results[r.job.jid] = r.W.cpu().numpy()
            except Exception as e:   # surfaced to the caller after the run
                errors.append(repr(e))
                with lock:
                    st["stop"] = True

        def pending_jobs(cls):
            return bool(pending_arrivals) or bool(queues[cls])

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
                                         stepped, ema, solo, z.plan_estimate_bytes, factor=self.factor,
                                         headroom=self.headroom,
                                         max_active=self.max_active, target=self.target,
                                         active_since=active_since, now=clock() - t0, session_s=self.session_s,
                                         compat=self.compat)
                    if cls is not None:
                        job = queues[cls].popleft()
                        took[cls] += 1
                        if took[cls] >= self.burst:   # the next job waits for a step with this set
                            stepped[cls] = False
                        if not classes.get(cls):
                            active_since[cls] = clock() - t0
                            ema.pop(cls, None)   # a new session measures afresh
                if job is None:
                    break
                need = z.plan_estimate_bytes(job.N, job.precision)
                ta = clock()
                admitting[0] += 1
                plan = z.Plan(job.N, job.precision)
                tb = clock()
                src = pinned.get(id(job.W0))   # initial states shared by jobs are pinned once
                if src is None:
                    src = torch.from_numpy(np.ascontiguousarray(job.W0)).pin_memory()
                    pinned[id(job.W0)] = src
                with torch.cuda.stream(upload):
                    W = src.to("cuda", non_blocking=True)
                upload.synchronize()
                admitting[0] -= 1
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
        gc.callbacks.remove(_gc_cb)
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
                           "max_resident": max_res[k],
                           "mean_resident": float(np.mean(res_hist[k])) if res_hist[k] else None,
                           "solo_ms": 1e3 * solo_step_s(solo, k, 1),   # one job of the class alone on the device
                           "p99_over_solo": _pct(v, 99) / (1e3 * solo_step_s(solo, k, 1))}
                          for k, v in lat.items()},
            "solo_calibration_ms": {f"N={k[0]},{'split' if k[1] == z.PRECISION_SPLIT else 'fp64'}":
                                    [1e3 * solo[k][0], 1e3 * solo[k][1]] for k in solo},
            "calibration_s": calib_s,
            "policy": {"max_active_classes": self.max_active, "latency_factor": self.factor,
                       "headroom": self.headroom,
                       "target_step_ms": None if self.target is None else self.target * 1e3,
                       "session_s": self.session_s, "compat": self.compat, "burst": self.burst},
            "queue_delay_s_p50": float(np.percentile(qdelay, 50)) if qdelay else None,
            "peak_admitted_bytes": st["peak"],
            "admit_plan_ms_mean": float(np.mean([a for a, _ in admit_times]) * 1e3) if admit_times else None,
            "admit_upload_ms_mean": float(np.mean([b for _, b in admit_times]) * 1e3) if admit_times else None,
            "step_time_ms_by_tag": _step_breakdown(step_log),
            "results": results,
        }
