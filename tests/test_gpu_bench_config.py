"""Parity at the benchmark's size and launch configuration (N = 4096, split form).

The product is checked on sampled rows the oracle side computes one by one
(row i of P W is P[i, :] @ W), for the tunings the benchmark runs; one whole
IsoMP step is checked against the oracle's step in tests/test_gpu_long_parity.py.
"""
import numpy as np
import pytest

from paper_2206_05466_gb300.inputs import vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402

N = 4096
H = 0.005
TUNINGS = [dict(),   # library defaults: persistent kernel, column-blocked order
           dict(exact_groups=2, tile_order=0),
           dict(exact_groups=2, no_persistent=1)]


@pytest.fixture(scope="module")
def operands():
    W = vorticity_w0(N, seed=0)
    plan = z.Plan(N, z.PRECISION_FP64)
    Wd = torch.from_numpy(W).cuda()
    Pd = torch.empty_like(Wd)
    z.zeitlin_stream_solve(plan, Wd, Pd)
    P = Pd.cpu().numpy()
    plan.close()
    return W, P


@pytest.mark.parametrize("tun", TUNINGS)
def test_split_product_sampled_rows(operands, tun):
    W, P = operands
    plan = z.Plan(N, z.PRECISION_SPLIT, **tun)
    C = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    z.zt_zgemm_skew(plan, torch.from_numpy(P).cuda(), torch.from_numpy(W).cuda(), C)
    got = C.cpu().numpy()
    plan.close()
    rows = np.unique(np.concatenate([[0, 1, 127, 128, N // 2, N - 129, N - 2, N - 1],
                                     np.random.default_rng(1).integers(0, N, 16)]))
    for i in rows:
        want = P[i, :] @ W
        err = np.linalg.norm(got[i] - want) / np.linalg.norm(want)
        assert err < 1e-11, (i, err)
