"""The serving admission policy (host logic, no GPU)."""
import collections
import dataclasses

from paper_2206_05466_gb300.serving import next_admission


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


def test_classes_in_order_of_their_head_arrival():
    q = _q(J(512, 0, 2.0), J(256, 1, 1.0), J(256, 1, 3.0))
    assert next_admission(q, {}, 0, 10**9, {}, {}, 0.1, est) == (256, 1)


def test_budget_skips_a_head_that_does_not_fit_but_not_when_nothing_is_resident():
    q = _q(J(4096, 0, 0.0), J(256, 0, 1.0))
    # nothing resident: the first head is admitted even above the budget
    assert next_admission(q, {}, 0, 1000, {}, {}, None, est) == (4096, 0)
    # something resident: the big head waits, the later small class goes first
    assert next_admission(q, {(512, 0): 1}, 500, 4000, {}, {}, None, est) == (256, 0)
    # nothing fits
    assert next_admission(q, {(512, 0): 1}, 3990, 4000, {}, {}, None, est) is None


def test_latency_target_gates_a_class_with_resident_jobs():
    q = _q(J(256, 1, 0.0))
    res = {(256, 1): 3}
    # no completed step since the last admission: wait
    assert next_admission(q, res, 0, 10**9, {(256, 1): False}, {(256, 1): 0.01}, 0.1, est) is None
    # stepped, but slower than the target: wait
    assert next_admission(q, res, 0, 10**9, {(256, 1): True}, {(256, 1): 0.2}, 0.1, est) is None
    # stepped and fast enough: admit
    assert next_admission(q, res, 0, 10**9, {(256, 1): True}, {(256, 1): 0.05}, 0.1, est) == (256, 1)
    # no target: footprint only
    assert next_admission(q, res, 0, 10**9, {}, {}, None, est) == (256, 1)


def test_an_empty_class_always_takes_its_head_job():
    q = _q(J(1024, 0, 0.0))
    assert next_admission(q, {(256, 1): 5}, 0, 10**9, {}, {(1024, 0): 9.9}, 0.1, est) == (1024, 0)


def test_empty_queues():
    assert next_admission(_q(), {}, 0, 10**9, {}, {}, 0.1, est) is None
