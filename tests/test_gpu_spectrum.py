"""Kinetic-energy spectrum on the device against the oracle (Sec. 4, basis of Sec. 3.2)."""
import numpy as np
import pytest

from oracle.spectrum import energy_spectrum, energy_spectrum_low
from paper_2206_05466_gb300.inputs import paper_omega, vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402


def _tol(W, N):
    l = np.arange(1, N)
    return 1e-12 * np.linalg.norm(W) ** 2 / (2.0 * l * (l + 1.0))


@pytest.mark.parametrize("N", [1, 2, 3, 5, 16, 33, 128, 129, 257, 600])
def test_spectrum_equals_oracle(N):
    W = vorticity_w0(N, seed=11)
    plan = z.Plan(N)
    E = z.zeitlin_energy_spectrum(plan, torch.from_numpy(W).cuda()).cpu().numpy()
    plan.close()
    want = energy_spectrum(W)
    assert E[0] == 0.0
    if N > 1:
        assert (np.abs(E[1:] - want[1:]) <= _tol(W, N)).all(), np.abs(E[1:] - want[1:]).max()
        L = min(N - 1, 10)
        low = energy_spectrum_low(W, L).astype(np.float64)
        assert np.abs(E[1:L + 1] / low[1:] - 1).max() < 1e-13


def test_spectrum_reads_only_the_lower_triangle():
    # W in su(N): the upper diagonals are -conj of the lower ones and are not read
    N = 70
    W = vorticity_w0(N, seed=2)
    plan = z.Plan(N)
    E = z.zeitlin_energy_spectrum(plan, torch.from_numpy(W).cuda()).cpu().numpy()
    Wc = W.copy()
    Wc[np.triu_indices(N, 1)] = 123.0 - 7.0j
    Ec = z.zeitlin_energy_spectrum(plan, torch.from_numpy(Wc).cuda()).cpu().numpy()
    plan.close()
    assert np.array_equal(E, Ec)
    assert (np.abs(E[1:] - energy_spectrum(W)[1:]) <= _tol(W, N)).all()


def test_spectrum_returns_the_coefficients_of_the_paper_initial_condition():
    N, lmax = 1024, 20
    om = paper_omega(lmax, lmin=2, seed=4)
    plan = z.Plan(N)
    B = z.Basis(plan, lmax)
    W = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    z.zeitlin_w_from_omega(B, torch.from_numpy(om).cuda(), W)
    E = z.zeitlin_energy_spectrum(plan, W).cpu().numpy()
    B.close()
    plan.close()
    want = np.zeros(N)
    for l in range(2, lmax + 1):
        want[l] = sum(abs(om[l * l + l + m]) ** 2 for m in range(-l, l + 1)) / (2 * l * (l + 1))
    assert np.abs(E - want).max() < 1e-12 * want.sum()


def test_spectrum_properties_at_n4096():
    N = 4096
    Wh = vorticity_w0(N, seed=0)
    W = torch.from_numpy(Wh).cuda()
    plan = z.Plan(N)
    E = z.zeitlin_energy_spectrum(plan, W)
    P = torch.empty_like(W)
    z.zeitlin_stream_solve(plan, W, P)
    H = 0.5 * torch.sum(P.transpose(0, 1) * W).item()   # (1/2) tr(P W)
    Eh = E.cpu().numpy()
    plan.close()
    l = np.arange(N)
    fro2 = float(np.sum(Wh.real ** 2 + Wh.imag ** 2))   # pairwise sum (a BLAS norm is ~1e-12 off here)
    assert E[0].item() == 0.0 and (Eh >= 0).all()
    assert abs(np.sum(2 * l * (l + 1) * Eh) - fro2) < 1e-12 * fro2      # Parseval
    # lowest modes, where rounded-block routes lose ~N^2 eps: the extended-precision oracle
    low = energy_spectrum_low(Wh, 8).astype(np.float64)
    assert np.abs(Eh[1:9] / low[1:] - 1).max() < 1e-13
    # Hamiltonian through the stream solve: the solve on blocks rounded to double is
    # conditioned like cond(T_0) ~ N^2/2 on the lowest modes, which dominate H
    assert abs(H.imag) < 1e-12 * abs(H.real)
    assert abs(Eh.sum() - H.real) < 0.5 * N * N * np.finfo(float).eps * abs(H.real)


def _on_diagonals(N, ms, seed):
    rng = np.random.default_rng(seed)
    W = np.zeros((N, N), complex)
    for m in ms:
        v = rng.standard_normal(N - m) + 1j * rng.standard_normal(N - m)
        W[np.arange(m, N), np.arange(0, N - m)] = v
        W[np.arange(0, N - m), np.arange(m, N)] = -np.conj(v)
    d = np.diag_indices(N)
    W[d] = 1j * W[d].imag
    return W


@pytest.mark.parametrize("N,ms", [(2048, [0, 1, 5, 64, 1024, 2046, 2047]),
                                  (4096, [2, 1500, 3000, 4000, 4094, 4095])])
def test_spectrum_element_wise_at_large_n(N, ms):
    # content on a few diagonals only, so that the oracle visits just those
    # blocks: element-wise at the benchmark sizes, including l close to large m
    # (the last entries of the diagonals, where the recurrence starts) and the
    # lowest l (extended-precision route)
    W = _on_diagonals(N, ms, seed=N)
    plan = z.Plan(N)
    E = z.zeitlin_energy_spectrum(plan, torch.from_numpy(W).cuda()).cpu().numpy()
    plan.close()
    want = energy_spectrum(W, diagonals=ms)
    L = 8
    assert (np.abs(E[L + 1:] - want[L + 1:]) <= _tol(W, N)[L:]).all(), np.abs(E[L + 1:] - want[L + 1:]).max()
    low = energy_spectrum_low(W, L).astype(np.float64)
    nz = low[1:] > 0
    if nz.any():
        assert np.abs(E[1:L + 1][nz] / low[1:][nz] - 1).max() < 1e-13
    assert np.all(E[1:L + 1][~nz] == 0.0) or not (~nz).any()
    assert E[ms[-1]] > 0 and E[ms[-2]] > 0   # l = N-1, N-2 blocks of size 1 and 2
