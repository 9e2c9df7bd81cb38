"""Bounded device waits of the split product kernel run out cleanly.

The kernel's producer thread can be told (testing-only tuning field
`debug_stall_loads`) to stop issuing operand loads after k - 1 of them, so
that the MMA thread's wait for the next load is a wait that nothing will
satisfy.  With a short limit (`wait_us`) the wait runs out, the CTA records
the timeout, waits for the copies and MMAs it had already issued, frees its
tensor memory and exits: the call returns ZT_ETIMEOUT, no fault, and the next
call on a fresh plan computes the right product.  Loads stop at once (k = 1,
nothing in flight) or after a few (k = 6: loads and MMAs in flight when the
wait runs out), in both forms of the kernel.
"""
import numpy as np
import pytest

import oracle
from paper_2206_05466_gb300.inputs import vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402

N = 256


def _operands():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    Y = vorticity_w0(N, seed=4)
    return X, Y


@pytest.mark.parametrize("stall", [1, 6])
@pytest.mark.parametrize("no_persistent", [0, 1])
def test_product_wait_runs_out(stall, no_persistent):
    X, Y = _operands()
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    C = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    plan = z.Plan(N, z.PRECISION_SPLIT, wait_us=20000, debug_stall_loads=stall, no_persistent=no_persistent)
    with pytest.raises(z.ZeitlinError) as ei:
        z.zt_zgemm_skew(plan, Xd, Yd, C)
    assert ei.value.code == z.ZT_ETIMEOUT
    plan.close()
    torch.cuda.synchronize()   # the context is still usable
    # the next plan, same operands: the right product
    good = z.Plan(N, z.PRECISION_SPLIT, no_persistent=no_persistent)
    z.zt_zgemm_skew(good, Xd, Yd, C)
    got = C.cpu().numpy()
    want = X @ Y
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12
    good.close()


def test_step_reports_timeout_then_recovers():
    W0 = vorticity_w0(N, seed=5)
    Wd = torch.from_numpy(W0.copy()).cuda()
    plan = z.Plan(N, z.PRECISION_SPLIT, wait_us=20000, debug_stall_loads=3)
    with pytest.raises(z.ZeitlinError) as ei:
        z.isomp_step(plan, Wd, 0.01)
    assert ei.value.code == z.ZT_ETIMEOUT
    plan.close()
    # afterwards a fresh plan steps the state as the oracle does
    a = z.Plan(N, z.PRECISION_SPLIT)
    Wa = torch.from_numpy(W0.copy()).cuda()
    info = z.isomp_step(a, Wa, 0.01)
    assert info["converged"]
    want, _ = oracle.isomp_step(W0, 0.01)
    got = Wa.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-10
    a.close()
