"""On-device Casimirs (zeitlin_casimirs) against the oracle, and their
conservation along IsoMP steps."""
import numpy as np
import pytest

import oracle
from paper_2206_05466_gb300.inputs import vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402

TOL = {z.PRECISION_FP64: 1e-12, z.PRECISION_SPLIT: 1e-10}


def _scale(W, k):
    lam = np.linalg.eigvalsh(-1j * W)
    return np.sum(np.abs(lam) ** k)


@pytest.mark.parametrize("precision", [z.PRECISION_FP64, z.PRECISION_SPLIT])
@pytest.mark.parametrize("N", [1, 2, 64, 300, 1024])
def test_casimirs_match_oracle(N, precision):
    W = vorticity_w0(N, seed=3 + N)
    plan = z.Plan(N, precision)
    got = z.zeitlin_casimirs(plan, torch.from_numpy(W).cuda())
    plan.close()
    want = oracle.casimirs(W, (2, 3, 4, 5))
    for k in (2, 3, 4, 5):
        sc = _scale(W, k)
        if sc == 0.0:   # N = 1: su(1) = {0}
            assert got[k] == 0
            continue
        assert abs(got[k] - want[k]) <= TOL[precision] * sc, (k, got[k], want[k])


@pytest.mark.parametrize("precision", [z.PRECISION_FP64, z.PRECISION_SPLIT])
def test_casimirs_conserved_along_steps(precision):
    N = 256
    W = torch.from_numpy(vorticity_w0(N, seed=11)).cuda()
    plan = z.Plan(N, precision)
    c0 = z.zeitlin_casimirs(plan, W)
    z.isomp_run(plan, W, 0.01, 10)
    c1 = z.zeitlin_casimirs(plan, W)
    plan.close()
    Wh = W.cpu().numpy()
    for k in (2, 3, 4, 5):
        assert abs(c1[k] - c0[k]) <= 1e-10 * _scale(Wh, k), k
