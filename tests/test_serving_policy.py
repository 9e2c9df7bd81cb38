"""The serving admission policy (host logic, no GPU)."""
import collections
import dataclasses

from paper_2206_05466_gb300.serving import next_admission, solo_step_s


@dataclasses.dataclass
class J:
    N: int
    precision: int
    arrival: float


def _q(*jobs):
    qs = collections.defaultdict(collections.deque)
    for j in jobs:
        qs[(j.N, j.precision)].append(j)
    return qs


def est(N, precision):
    return N * 10


SOLO = collections.defaultdict(lambda: (0.010, 0.002))   # 10 ms for one job, +2 ms per further job


def pick(q, res, used=0, budget=10**9, stepped=None, ema=None, **kw):
    return next_admission(q, res, used, budget, stepped or {}, ema or {}, SOLO, est, **kw)


def test_solo_model():
    assert abs(solo_step_s({"c": (0.01, 0.002)}, "c", 1) - 0.01) < 1e-15
    assert abs(solo_step_s({"c": (0.01, 0.002)}, "c", 4) - 0.016) < 1e-15


def test_classes_in_order_of_their_head_arrival():
    q = _q(J(512, 0, 2.0), J(256, 1, 1.0), J(256, 1, 3.0))
    assert pick(q, {}) == (256, 1)


def test_budget_skips_a_head_that_does_not_fit_but_not_when_nothing_is_resident():
    q = _q(J(4096, 0, 0.0), J(256, 0, 1.0))
    # nothing resident: the first head is admitted even above the budget
    assert pick(q, {}, 0, 1000) == (4096, 0)
    # something resident: the big head waits, the later small class goes first
    assert pick(q, {(512, 0): 1}, 500, 4000) == (256, 0)
    # nothing fits
    assert pick(q, {(512, 0): 1}, 3990, 4000) is None


def test_at_most_two_classes_resident():
    q = _q(J(256, 1, 0.0), J(1024, 0, 1.0))
    res = {(512, 0): 2, (2048, 1): 1}
    assert pick(q, res) is None                     # two classes active: no third
    assert pick(q, res, max_active=3) == (256, 1)
    assert pick(q, {(512, 0): 2}) == (256, 1)       # one active: a second may start


def test_latency_gates_a_resident_class():
    c = (256, 1)
    q = _q(J(256, 1, 0.0))
    res = {c: 3}   # solo with one job: 10 ms; the gate: 0.8 x 2 x 10 ms = 16 ms
    # no completed step since the last admission: wait
    assert pick(q, res, stepped={c: False}, ema={c: 0.012}) is None
    # stepped, but the batch already takes more than the gate: wait
    assert pick(q, res, stepped={c: True}, ema={c: 0.017}) is None
    # stepped, below the gate: admit
    assert pick(q, res, stepped={c: True}, ema={c: 0.013}) == c
    # the headroom is a parameter
    assert pick(q, res, stepped={c: True}, ema={c: 0.017}, headroom=0.9) == c
    # the absolute target bounds the solo step time with one more job (16 ms)
    assert pick(q, res, stepped={c: True}, ema={c: 0.013}, target=0.015) is None
    assert pick(q, res, stepped={c: True}, ema={c: 0.013}, target=0.017) == c
    # an empty class always takes its head job, whatever the target
    assert pick(_q(J(1024, 0, 0.0)), {}, target=0.001) == (1024, 0)


def test_sessions_rotate_classes():
    c, other = (256, 1), (512, 0)
    q = _q(J(256, 1, 5.0), J(512, 0, 1.0))
    res = {c: 2, (1024, 0): 1}   # two active classes; `other` waits for a place
    kw = dict(stepped={c: True}, ema={c: 0.011}, session_s=20.0)
    # within its session the active class keeps admitting
    assert pick(q, res, active_since={c: 0.0}, now=10.0, **kw) == c
    # past its session, with another class waiting, it admits no more
    assert pick(q, res, active_since={c: 0.0}, now=30.0, **kw) is None
    # ... but it does when nobody else waits
    q2 = _q(J(256, 1, 5.0))
    assert pick(q2, res, active_since={c: 0.0}, now=30.0, **kw) == c


def test_empty_queues():
    assert pick(_q(), {}) is None


def test_no_latency_gate_admits_by_footprint_and_class_count():
    c = (40, 1)
    q = _q(J(40, 1, 0.0), J(40, 1, 0.0))
    assert pick(q, {c: 1}, factor=None, target=None) == c
    assert pick(q, {c: 1}, factor=None, target=None, stepped={c: False}) == c


def test_compatibility_keeps_light_and_heavy_classes_apart():
    solo = {(256, 1): (0.0015, 0.0), (2048, 0): (0.36, 0.3), (512, 1): (0.003, 0.0)}
    q = _q(J(2048, 0, 0.0), J(512, 1, 1.0))
    res = {(256, 1): 2}
    got = next_admission(q, res, 0, 10**9, {}, {}, solo, est, compat=8.0)
    assert got == (512, 1)            # the heavy head waits; the compatible class goes first
    assert next_admission(_q(J(2048, 0, 0.0)), res, 0, 10**9, {}, {}, solo, est, compat=8.0) is None
    assert next_admission(_q(J(2048, 0, 0.0)), res, 0, 10**9, {}, {}, solo, est, compat=None) == (2048, 0)
    assert next_admission(_q(J(2048, 0, 0.0)), {}, 0, 10**9, {}, {}, solo, est, compat=8.0) == (2048, 0)


def test_calibrated_cost_of_one_more_job_is_gated_too():
    # heavy per-job cost: one job 50 ms, +25 ms per further job; the gate 0.8 x 2 x 50 = 80 ms
    c = (1024, 0)
    solo = {c: (0.050, 0.025)}
    q = _q(J(1024, 0, 0.0))
    kw = dict(stepped={c: True}, ema={c: 0.050})
    assert next_admission(q, {c: 1}, 0, 10**9, solo=solo, estimate=est, **kw) == c       # 2 jobs: 75 ms
    kw = dict(stepped={c: True}, ema={c: 0.075})
    assert next_admission(q, {c: 2}, 0, 10**9, solo=solo, estimate=est, **kw) is None    # 3 jobs: 100 ms
