"""Continuous-batching serving loop: each result is the same alone and in the mix.

Jobs of different N and precision arrive over time, are admitted by device
footprint and class step latency and stepped together in batched steps; every job's final state must
equal, bit for bit, the state of the same job stepped alone with isomp_step
(the grouped kernels run each instance's arithmetic unchanged).
"""
import numpy as np
import pytest

from paper_2206_05466_gb300.inputs import vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import serving  # noqa: E402
from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402


def _jobs():
    spec = [(32, 4, z.PRECISION_SPLIT, 0.0), (48, 6, z.PRECISION_FP64, 0.0), (64, 3, z.PRECISION_SPLIT, 0.005),
            (40, 5, z.PRECISION_SPLIT, 0.01), (64, 2, z.PRECISION_FP64, 0.02), (33, 7, z.PRECISION_SPLIT, 0.03)]
    return [serving.Job(jid=k, N=N, nsteps=n, h=0.01, precision=prec, arrival=t, W0=vorticity_w0(N, seed=20 + k))
            for k, (N, n, prec, t) in enumerate(spec)]


def _alone(job):
    plan = z.Plan(job.N, job.precision)
    W = torch.from_numpy(job.W0.copy()).cuda()
    for _ in range(job.nsteps):
        z.isomp_step(plan, W, job.h)
    out = W.cpu().numpy()
    plan.close()
    return out


def test_results_alone_equal_results_in_the_mix():
    graph = False
    jobs = _jobs()
    budget = sum(z.plan_estimate_bytes(j.N, j.precision) for j in jobs[:3])   # forces queueing
    rep = serving.Server(budget, graph=graph).run(jobs, keep_results=True)
    assert rep["jobs_completed"] == len(jobs)
    assert rep["job_steps"] == sum(j.nsteps for j in jobs)
    assert rep["peak_admitted_bytes"] <= budget
    assert rep["step_latency_ms_p99"] >= rep["step_latency_ms_p50"] > 0
    for j in jobs:
        assert np.array_equal(rep["results"][j.jid], _alone(j)), j.jid


def test_latency_target_admits_one_job_per_class_at_a_time():
    """A target no step can meet: each class keeps exactly one resident job, the
    rest wait in the class's queue; at most two classes are resident at once;
    results are unchanged."""
    jobs = _jobs()
    rep = serving.Server(1 << 40, target_step_ms=1e-6).run(jobs, keep_results=True)
    assert rep["jobs_completed"] == len(jobs)
    assert all(c["max_resident"] == 1 for c in rep["per_class"].values()), rep["per_class"]
    for j in jobs:
        assert np.array_equal(rep["results"][j.jid], _alone(j)), j.jid


def test_footprint_only_admission_batches_jobs_of_a_class():
    """Without a latency target, jobs of one class that are all waiting at the
    start are admitted together and stepped as one batch."""
    jobs = [serving.Job(jid=k, N=40, nsteps=40, h=0.01, precision=z.PRECISION_SPLIT, arrival=0.0,
                        W0=vorticity_w0(40, seed=40 + k)) for k in range(4)]
    rep = serving.Server(1 << 40, target_step_ms=None, latency_factor=None).run(jobs, keep_results=True)
    assert rep["jobs_completed"] == 4
    assert rep["per_class"]["N=40,split"]["max_resident"] == 4
    assert rep["batched_steps"] < rep["job_steps"]
    for j in jobs:
        assert np.array_equal(rep["results"][j.jid], _alone(j)), j.jid
