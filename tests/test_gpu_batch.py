"""Grouped (batched) IsoMP steps over ensembles of independent instances.

A batched step must advance every instance exactly as isomp_step does on its
own -- bit for bit, since the grouped kernels run the same per-instance
arithmetic in the same order -- for any mix of N and precision, with
per-instance convergence (instances that converge early are masked off).
"""
import numpy as np
import pytest

import oracle
from paper_2206_05466_gb300.inputs import vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


MIX = [(64, z.PRECISION_SPLIT, 0.01), (130, z.PRECISION_SPLIT, 0.005), (33, z.PRECISION_SPLIT, -0.02),
       (256, z.PRECISION_SPLIT, 0.01), (64, z.PRECISION_FP64, 0.01), (100, z.PRECISION_FP64, 0.03),
       (1, z.PRECISION_SPLIT, 0.01), (2, z.PRECISION_FP64, 0.2)]


def _singles(cases, nsteps, seed0=0):
    out = []
    for k, (N, prec, h) in enumerate(cases):
        plan = z.Plan(N, prec)
        W = _cuda(vorticity_w0(N, seed=seed0 + k))
        iters = []
        for _ in range(nsteps):
            iters.append(z.isomp_step(plan, W, h)["iters"])
        out.append((W.cpu().numpy(), iters))
        plan.close()
    return out


def _batch(cases, seed0=0, graph=False):
    plans = [z.Plan(N, prec) for N, prec, _ in cases]
    Ws = [_cuda(vorticity_w0(N, seed=seed0 + k)) for k, (N, _, _) in enumerate(cases)]
    b = z.Batch(plans, Ws, [h for _, _, h in cases])
    if graph:
        b.set_graph(True)
    return b, plans, Ws


@pytest.mark.parametrize("graph", [False, True])
def test_batched_steps_equal_single_steps_bitwise(graph):
    nsteps = 3
    want = _singles(MIX, nsteps)
    b, plans, Ws = _batch(MIX, graph=graph)
    iters = [[] for _ in MIX]
    for _ in range(nsteps):
        rc, st = b.step()
        assert rc == z.ZT_OK
        for k, x in enumerate(st):
            iters[k].append(x["iters"])
    for k, (W, (Wref, it_ref)) in enumerate(zip(Ws, want)):
        assert np.array_equal(W.cpu().numpy(), Wref), MIX[k]
        assert iters[k] == it_ref, (MIX[k], iters[k], it_ref)
    assert b.launch_count() > 0


def test_batched_matches_oracle_and_masks_converged_members():
    # very different step sizes converge after different sweep counts
    cases = [(48, z.PRECISION_SPLIT, 1e-4), (48, z.PRECISION_SPLIT, 0.05), (40, z.PRECISION_FP64, 0.08)]
    b, plans, Ws = _batch(cases, seed0=10)
    rc, st = b.step()
    assert rc == z.ZT_OK
    its = [x["iters"] for x in st]
    assert its[0] < its[1], its
    for k, (N, prec, h) in enumerate(cases):
        want, info = oracle.isomp_step(vorticity_w0(N, seed=10 + k), h)
        got = Ws[k].cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-10
        assert its[k] == info.iters or abs(its[k] - info.iters) <= 1


def test_batched_nonfinite_member_is_isolated():
    cases = [(32, z.PRECISION_SPLIT, 0.01), (32, z.PRECISION_SPLIT, 0.01)]
    plans = [z.Plan(N, prec) for N, prec, _ in cases]
    W0 = vorticity_w0(32, seed=1)
    bad = W0.copy()
    bad[4, 2] = np.nan
    Ws = [_cuda(W0), _cuda(bad)]
    b = z.Batch(plans, Ws, [0.01, 0.01])
    with pytest.raises(z.ZeitlinError) as e:
        b.step()
    assert e.value.code == z.ZT_ENONFINITE
    want, _ = oracle.isomp_step(W0, 0.01)
    got = Ws[0].cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-10


def test_run_batched_totals():
    cases = [(64, z.PRECISION_SPLIT, 0.01), (96, z.PRECISION_SPLIT, 0.01)]
    b, plans, Ws = _batch(cases, seed0=3)
    r = b.run(4)
    assert r["steps"] == 4 and r["all_converged"] and r["total_iters"] >= 4 * 2 * 2


def test_multi_step_large_grids():
    # N = 2048: the update and product grids span several waves of CTAs, so a
    # state flag written by one CTA must never gate the rest of its own launch.
    N, h, nsteps = 2048, 0.005, 3
    W0 = vorticity_w0(N, seed=0)
    outs = {}
    for prec in (z.PRECISION_SPLIT, z.PRECISION_FP64):
        plan = z.Plan(N, prec)
        W = _cuda(W0)
        for _ in range(nsteps):
            info = z.isomp_step(plan, W, h)
            assert info["converged"]
        outs[prec] = W.cpu().numpy()
        plan.close()
    a, b = outs[z.PRECISION_SPLIT], outs[z.PRECISION_FP64]
    assert np.all(np.isfinite(a))
    want, _ = oracle.isomp_run(W0, h, nsteps)   # both forms against the oracle, not each other
    assert np.linalg.norm(a - want) / np.linalg.norm(want) < 1e-10
    assert np.linalg.norm(b - want) / np.linalg.norm(want) < 1e-11
    # the same instance inside a batch, next to a smaller one, for the same steps
    plans = [z.Plan(N, z.PRECISION_SPLIT), z.Plan(512, z.PRECISION_SPLIT)]
    Ws = [_cuda(W0), _cuda(vorticity_w0(512, seed=1))]
    bt = z.Batch(plans, Ws, [h, h])
    for _ in range(nsteps):
        bt.step()
    assert np.array_equal(Ws[0].cpu().numpy(), a)
