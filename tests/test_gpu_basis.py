"""Quantised basis on the device against the oracle (Sec. 3.2, Eqs. 10-12)."""
import numpy as np
import pytest

from oracle import basis as ob
from paper_2206_05466_gb300.inputs import paper_omega, vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402


@pytest.mark.parametrize("N,lmax,ls", [(1, 0, None), (2, 1, None), (5, 4, None), (12, 11, None),
                                       (64, 63, [0, 1, 2, 31, 62, 63])])
def test_basis_vectors_equal_the_3j_route(N, lmax, ls):
    plan = z.Plan(N)
    B = z.Basis(plan, lmax)
    for l in (ls if ls is not None else range(lmax + 1)):
        for m in range(l + 1):
            want = np.diag(ob.that_lm(N, l, m), -m)
            assert np.abs(B.vector(l, m) - want).max() < 1e-13, (l, m)
    B.close()
    plan.close()


@pytest.mark.parametrize("N,lmax", [(129, 24), (512, 24), (1024, 16)])
def test_basis_vectors_equal_the_lapack_route(N, lmax):
    plan = z.Plan(N)
    B = z.Basis(plan, lmax)
    for l in range(lmax + 1):
        for m in range(l + 1):
            want = np.diag(ob.that_lm_eig(N, l, m), -m)
            assert np.abs(B.vector(l, m) - want).max() < 1e-12, (l, m)
    B.close()
    plan.close()


@pytest.mark.parametrize("N,lmax", [(7, 6), (16, 9)])
def test_w_from_omega_equals_oracle(N, lmax):
    om = paper_omega(lmax, lmin=0, seed=N)
    om[0] = 0.0
    plan = z.Plan(N)
    B = z.Basis(plan, lmax)
    W = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    z.zeitlin_w_from_omega(B, torch.from_numpy(om).cuda(), W)
    got = W.cpu().numpy()
    B.close()
    plan.close()
    want = ob.w_from_omega(N, om, lmax)
    assert np.abs(got - want).max() < 1e-13
    assert np.array_equal(got, -got.conj().T)   # exactly skew-Hermitian


@pytest.mark.parametrize("N,lmax", [(256, 20), (1024, 32)])
def test_omega_round_trip_and_paper_initial_condition(N, lmax):
    om = paper_omega(lmax, lmin=2, seed=3)
    plan = z.Plan(N)
    B = z.Basis(plan, lmax)
    omd = torch.from_numpy(om).cuda()
    W = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    z.zeitlin_w_from_omega(B, omd, W)
    back = torch.empty_like(omd)
    z.zeitlin_omega_from_w(B, W, back)
    assert np.abs(back.cpu().numpy() - om).max() < 1e-12 * np.abs(om).max()
    Wh = W.cpu().numpy()
    assert np.array_equal(Wh, -Wh.conj().T)
    # tr T^_l0 = 0 for l > 0: the trace is rounding of N diagonal terms
    assert abs(np.trace(Wh)) < 1e-14 * N * np.abs(np.diag(Wh)).max() * lmax
    # the paper's initial condition steps like any other vorticity matrix
    W /= float(np.linalg.norm(Wh, 2))
    info = z.isomp_step(plan, W, 0.01)
    assert info["converged"]
    B.close()
    plan.close()


def test_basis_outlives_its_plan():
    N, lmax = 33, 8
    plan = z.Plan(N)
    B = z.Basis(plan, lmax)
    want = B.vector(5, 2)
    plan.close()   # the plan is read only while the basis is created
    om = torch.from_numpy(paper_omega(lmax, seed=1)).cuda()
    W = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    z.zeitlin_w_from_omega(B, om, W)
    assert np.array_equal(B.vector(5, 2), want)
    B.close()
    assert np.abs(W.cpu().numpy() - ob.w_from_omega(N, om.cpu().numpy(), lmax)).max() < 1e-13


def test_basis_argument_checks():
    plan = z.Plan(8)
    for bad in (8, -1):
        with pytest.raises(z.ZeitlinError):
            z.Basis(plan, bad)
    B = z.Basis(plan, 3)
    for l, m in ((2, 3), (4, 0), (1, -1)):
        with pytest.raises(z.ZeitlinError):
            B.vector(l, m)
    W = torch.empty((8, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        z.zeitlin_w_from_omega(B, torch.zeros(15, dtype=torch.complex128, device="cuda"), W)
    B.close()
    plan.close()


@pytest.mark.parametrize("N,lmax,route", [(40, 12, "3j"), (256, 20, "eig")])
def test_omega_from_w_projects_a_full_matrix(N, lmax, route):
    # W with content at every l <= N-1 (the seeded recipe): omega_from_w must
    # return the projection onto the l <= lmax span, omega_lm = -i tr(T^_lm^H W),
    # not just invert w_from_omega on that span
    W = vorticity_w0(N, seed=9)
    plan = z.Plan(N)
    B = z.Basis(plan, lmax)
    om = torch.empty((lmax + 1) ** 2, dtype=torch.complex128, device="cuda")
    z.zeitlin_omega_from_w(B, torch.from_numpy(W).cuda(), om)
    got = om.cpu().numpy()
    B.close()
    plan.close()
    want = ob.omega_from_w(N, W, lmax, route=route)
    assert np.abs(got - want).max() < 1e-12 * np.sqrt(N) * np.abs(W).max()
    # the part of W off the span is really there: the projection loses norm
    assert np.linalg.norm(want) < 0.999 * np.linalg.norm(W)
