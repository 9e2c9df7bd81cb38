"""The fixed point's first iterate (Eq. 9): extrapolated along the trajectory.

A plan that advanced the same W with the same h in its previous step starts the
next step's iteration from W_n + (W_n - W_{n-1})/2 instead of W_n.  The fixed
point is the same (within tol); the GPU step is compared with the oracle started
from the same first iterate (same sweep count) and from W_n, and the history is
dropped whenever W or h changes.
"""
import numpy as np
import pytest

import oracle
from paper_2206_05466_gb300.inputs import vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [(z.PRECISION_FP64, 1e-11), (z.PRECISION_SPLIT, 1e-10)])
def test_extrapolated_steps_match_the_oracle(prec, tol):
    N, h = 96, 0.005
    W0 = vorticity_w0(N, seed=21)
    plan = z.Plan(N, prec)
    W = torch.from_numpy(W0.copy()).cuda()
    prev = W0
    for n in range(4):
        cur = W.cpu().numpy()
        info = z.isomp_step(plan, W, h)
        got = W.cpu().numpy()
        first = cur if n == 0 else cur + 0.5 * (cur - prev)
        same, st_same = oracle.isomp_step(cur, h, Wt0=first)
        plain, st_plain = oracle.isomp_step(cur, h)
        assert info["converged"]
        assert abs(info["iters"] - st_same.iters) <= 1, (n, info["iters"], st_same.iters)
        assert _rel(got, same) <= tol and _rel(got, plain) <= tol
        if n > 0:
            assert st_same.iters <= st_plain.iters
        prev = cur
    plan.close()


def test_extrapolation_saves_a_sweep_at_the_benchmark_step_size():
    N, h = 512, 0.005
    W0 = vorticity_w0(N, seed=0)
    a = z.Plan(N, z.PRECISION_SPLIT)
    b = z.Plan(N, z.PRECISION_SPLIT, first_iterate=z.FIRST_WN)
    Wa = torch.from_numpy(W0.copy()).cuda()
    Wb = torch.from_numpy(W0.copy()).cuda()
    ia, ib = [], []
    for _ in range(4):
        ia.append(z.isomp_step(a, Wa, h)["iters"])
        ib.append(z.isomp_step(b, Wb, h)["iters"])
    assert ia[0] == ib[0]                       # no history yet
    assert all(x <= y for x, y in zip(ia[1:], ib[1:])) and sum(ia[1:]) < sum(ib[1:]), (ia, ib)
    assert _rel(Wa.cpu().numpy(), Wb.cpu().numpy()) < 1e-12
    a.close()
    b.close()


def test_history_is_dropped_for_another_w_or_h():
    N, h = 80, 0.01
    W1 = vorticity_w0(N, seed=1)
    W2 = vorticity_w0(N, seed=2)
    p = z.Plan(N, z.PRECISION_SPLIT)
    A = torch.from_numpy(W1.copy()).cuda()
    for _ in range(2):
        z.isomp_step(p, A, h)
    # another buffer: the step must equal a fresh plan's first step, bit for bit
    B = torch.from_numpy(W2.copy()).cuda()
    z.isomp_step(p, B, h)
    q = z.Plan(N, z.PRECISION_SPLIT)
    Bq = torch.from_numpy(W2.copy()).cuda()
    z.isomp_step(q, Bq, h)
    assert np.array_equal(B.cpu().numpy(), Bq.cpu().numpy())
    # the same buffer with another step size: no history either
    C = B.clone()
    z.isomp_step(p, B, 2 * h)
    r = z.Plan(N, z.PRECISION_SPLIT)
    z.isomp_step(r, C, 2 * h)
    assert np.array_equal(B.cpu().numpy(), C.cpu().numpy())
    for x in (p, q, r):
        x.close()


def test_first_iterate_wn_follows_the_oracle_sweep_for_sweep():
    N, h = 64, 0.01
    W = torch.from_numpy(vorticity_w0(N, seed=5)).cuda()
    p = z.Plan(N, z.PRECISION_FP64, first_iterate=z.FIRST_WN)
    for _ in range(3):
        cur = W.cpu().numpy()
        info = z.isomp_step(p, W, h)
        want, st = oracle.isomp_step(cur, h)
        assert info["iters"] == st.iters
        assert _rel(W.cpu().numpy(), want) <= 1e-11
    p.close()


def test_reset_history_gives_the_w_n_start():
    N, h = 72, 0.01
    W0 = vorticity_w0(N, seed=9)
    p = z.Plan(N, z.PRECISION_SPLIT)
    A = torch.from_numpy(W0.copy()).cuda()
    for _ in range(2):
        z.isomp_step(p, A, h)
    p.reset_history()
    B = A.clone()
    z.isomp_step(p, A, h)
    q = z.Plan(N, z.PRECISION_SPLIT)
    z.isomp_step(q, B, h)
    assert np.array_equal(A.cpu().numpy(), B.cpu().numpy())
    p.close()
    q.close()
