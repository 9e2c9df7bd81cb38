"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerances:
  * Laplacian apply, stream solve: FP64 work of O(1) operations per element,
    compared element by element at 1e-13 relative to the largest entry.
  * FP64 product: relative Frobenius 1e-13 (K-term FP64 sums, K <= 2N).
  * IsoMP step, FP64 form: relative Frobenius error of W <= 1e-11 after every
    step of the trajectory.
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


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


SIZES = [1, 2, 3, 5, 31, 32, 33, 64, 100, 257]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    z.load()
    yield


@pytest.mark.parametrize("N", SIZES)
def test_laplacian_apply(N):
    rng = np.random.default_rng(N)
    P = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    plan = z.Plan(N)
    Wd = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    z.zeitlin_laplacian_apply(plan, _cuda(P), Wd)
    got = Wd.cpu().numpy()
    want = oracle.laplacian_apply(P)
    assert np.abs(got - want).max() <= 1e-13 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("N", SIZES + [1024])
def test_stream_solve(N):
    W = vorticity_w0(N, seed=N)
    plan = z.Plan(N)
    Pd = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    z.zeitlin_stream_solve(plan, _cuda(W), Pd)
    got = Pd.cpu().numpy()
    want = oracle.stream_solve(W)
    assert np.abs(got - want).max() <= 1e-13 * max(1e-300, np.abs(want).max())
    assert np.abs(got + got.conj().T).max() == 0.0


def test_stream_solve_reads_only_lower_triangle():
    N = 70
    W = vorticity_w0(N, seed=1)
    Wj = W.copy()
    Wj[np.triu_indices(N, 1)] = np.nan
    plan = z.Plan(N)
    Pd = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    z.zeitlin_stream_solve(plan, _cuda(Wj), Pd)
    assert np.abs(Pd.cpu().numpy() - oracle.stream_solve(W)).max() < 1e-13


@pytest.mark.parametrize("N", [1, 2, 17, 64, 65, 130, 256])
def test_zgemm_skew_fp64(N):
    rng = np.random.default_rng(100 + N)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    Y = vorticity_w0(N, seed=3)
    plan = z.Plan(N)
    Cd = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    z.zt_zgemm_skew(plan, _cuda(X), _cuda(Y), Cd)
    want = X @ Y
    assert _rel(Cd.cpu().numpy(), want) < 1e-13


def test_isomp_trajectory_fp64_n64():
    # Plain FP64, N=64, h=0.01, 100 steps, tol 1e-12, maxit 50: every step.
    N, h, steps = 64, 0.01, 100
    W0 = vorticity_w0(N, seed=0)
    plan = z.Plan(N, z.PRECISION_FP64)
    Wd = _cuda(W0)
    Wo = W0.copy()
    worst = 0.0
    for n in range(steps):
        info = z.isomp_step(plan, Wd, h)
        Wo, oi = oracle.isomp_step(Wo, h)
        err = _rel(Wd.cpu().numpy(), Wo)
        worst = max(worst, err)
        assert err <= 1e-11, (n, err)
        assert abs(info["iters"] - oi.iters) <= 1
    assert worst <= 1e-11


@pytest.mark.parametrize("N,h", [(1, 0.01), (2, 0.3), (3, 0.01), (33, -0.02)])
def test_isomp_small_and_ragged(N, h):
    W0 = vorticity_w0(N, seed=5)
    plan = z.Plan(N)
    Wd = _cuda(W0)
    for _ in range(3):
        z.isomp_step(plan, Wd, h)
    want, _ = oracle.isomp_run(W0, h, 3)
    got = Wd.cpu().numpy()
    if np.linalg.norm(want) == 0:
        assert np.abs(got).max() == 0
    else:
        assert _rel(got, want) <= 1e-11


def test_isomp_run_matches_steps_bitwise():
    N, h = 96, 0.01
    W0 = vorticity_w0(N, seed=9)
    plan = z.Plan(N)
    Wa = _cuda(W0)
    r = z.isomp_run(plan, Wa, h, 5)
    assert r["steps"] == 5 and r["all_converged"]
    Wb = _cuda(W0)
    for _ in range(5):
        z.isomp_step(plan, Wb, h)
    assert torch.equal(Wa, Wb)


def test_reuse_final_mode():
    N, h = 64, 0.01
    W0 = vorticity_w0(N, seed=4)
    plan = z.Plan(N, final_mode=z.FINAL_REUSE)
    Wd = _cuda(W0)
    z.isomp_step(plan, Wd, h)
    want, _ = oracle.isomp_step(W0, h, final="reuse")
    assert _rel(Wd.cpu().numpy(), want) <= 1e-11


def test_not_converged_status_and_result_written():
    N, h = 64, 0.01
    W0 = vorticity_w0(N, seed=0)
    plan = z.Plan(N)
    Wd = _cuda(W0)
    info = z.isomp_step(plan, Wd, h, maxit=1, allow_not_converged=True)
    assert info["status"] == z.ZT_NOT_CONVERGED and info["iters"] == 1 and not info["converged"]
    want, _ = oracle.isomp_step(W0, h, maxit=1)
    assert _rel(Wd.cpu().numpy(), want) <= 1e-11


def test_nonfinite_input_is_reported():
    N = 40
    W0 = vorticity_w0(N, seed=0)
    W0[5, 3] = np.nan
    plan = z.Plan(N)
    with pytest.raises(z.ZeitlinError) as e:
        z.isomp_step(plan, _cuda(W0), 0.01)
    assert e.value.code == z.ZT_ENONFINITE
    # the plan stays usable
    Wd = _cuda(vorticity_w0(N, seed=1))
    z.isomp_step(plan, Wd, 0.01)


def test_isomp_n1024_first_steps_fp64():
    N, h = 1024, 0.01
    W0 = vorticity_w0(N, seed=0)
    plan = z.Plan(N)
    Wd = _cuda(W0)
    Wo = W0
    for n in range(2):
        z.isomp_step(plan, Wd, h)
        Wo, _ = oracle.isomp_step(Wo, h)
        assert _rel(Wd.cpu().numpy(), Wo) <= 1e-11
