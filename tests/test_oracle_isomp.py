"""Pins of the oracle's IsoMP step (CPU only).

The step is an iteration, so it is pinned by what the paper and the algebra
fix rather than by stored trajectories:
  * both lines of Eq. 8, re-evaluated with explicit products and a
    stream matrix from the dense spin-Casimir pseudo-inverse;
  * steady states (W inside one l-eigenspace, and every W at N = 2);
  * second-order agreement with an independent RK4 integration of
    Eq. 6 (this fixes the direction of time);
  * reversibility, isospectrality and Casimir conservation (Sec. 2);
  * preservation of su(N).
A few tests plant a mistake in a copy of the step and check that the pins
catch it.
"""
import numpy as np
import pytest

import oracle
from oracle import zeitlin as oz
from paper_2206_05466_gb300.inputs import vorticity_w0
from tests import _spin


def _isomp_lines(Wn, Wnp1, Wt, N, h):
    """Residuals of both lines of Eq. 8 with an independent stream matrix."""
    Pt = (_spin.dense_pseudo_inverse(N) @ Wt.reshape(-1)).reshape(N, N)
    I = np.eye(N)
    first = (I - h / 2 * Pt) @ Wt @ (I + h / 2 * Pt)
    second = (I + h / 2 * Pt) @ Wt @ (I - h / 2 * Pt)
    return np.abs(first - Wn).max(), np.abs(second - Wnp1).max()


@pytest.mark.parametrize("N,h", [(6, 0.05), (9, 0.1), (12, -0.07)])
def test_both_lines_of_isomp_hold(N, h):
    Wn = vorticity_w0(N, seed=3)
    Wnp1, info = oracle.isomp_step(Wn, h, tol=1e-14, maxit=100)
    assert info.converged
    e1, e2 = _isomp_lines(Wn, Wnp1, info.Wt, N, h)
    assert e1 < 1e-13 and e2 < 1e-13, (e1, e2)


def _step_dropped_h2(Wn, h, tol=1e-14, maxit=100):
    # planted mistake: the h^2/4 term of Eq. 9 is dropped
    Wt = Wn.copy()
    for _ in range(maxit):
        Pt = oz.stream_solve(Wt)
        A = Pt @ Wt
        Wnew = Wn + h / 2 * (A - A.conj().T)
        done = np.linalg.norm(Wnew - Wt) < tol
        Wt = Wnew
        if done:
            break
    Pt = oz.stream_solve(Wt)
    A = Pt @ Wt
    B = A @ Pt
    return Wt + h / 2 * (A - A.conj().T) - h * h / 4 * B, Wt


def _step_wrong_sign(Wn, h):
    # planted mistake: commutator taken as Wt Pt - Pt Wt
    W, info = oracle.isomp_step(Wn, -h, tol=1e-14, maxit=100)
    return W, info.Wt


def test_planted_mistakes_fail_the_isomp_pin():
    N, h = 9, 0.1
    Wn = vorticity_w0(N, seed=3)
    W1, Wt1 = _step_dropped_h2(Wn, h)
    assert max(_isomp_lines(Wn, W1, Wt1, N, h)) > 1e-8
    W2, Wt2 = _step_wrong_sign(Wn, h)
    assert max(_isomp_lines(Wn, W2, Wt2, N, h)) > 1e-8


def test_steady_states():
    # N = 2: su(2) is the single l = 1 eigenspace, so [P, W] = 0.
    W = _spin.random_su(2, 0)
    W1, info = oracle.isomp_step(W, 0.3)
    np.testing.assert_allclose(W1, W, atol=1e-15)
    # any N: W spanned by i S_a (l = 1) is a steady state.
    N = 16
    S1, S2, S3 = _spin.spin_matrices(N)
    W = 1j * (0.2 * S1 + 0.5 * S2 - 0.1 * S3)
    W /= np.abs(np.linalg.eigvalsh(-1j * W)).max()
    W1, info = oracle.isomp_step(W, 0.05)
    np.testing.assert_allclose(W1, W, atol=1e-14)
    # the midpoint matrix itself moves (h^2/4 Pt Wt Pt != 0): Wt != W_n
    assert np.abs(info.Wt - W).max() > 1e-6


def _rk4_reference(W0, t, nsub):
    """Independent integration of dW/dt = [P, W], Delta_N P = W (Eq. 6)."""
    N = W0.shape[0]
    Linv = _spin.dense_pseudo_inverse(N)

    def f(W):
        P = (Linv @ W.reshape(-1)).reshape(N, N)
        return P @ W - W @ P

    W = W0.copy()
    dt = t / nsub
    for _ in range(nsub):
        k1 = f(W)
        k2 = f(W + dt / 2 * k1)
        k3 = f(W + dt / 2 * k2)
        k4 = f(W + dt * k3)
        W = W + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return W


def test_second_order_agreement_with_rk4():
    N = 8
    W0 = vorticity_w0(N, seed=7) * 3.0
    errs = []
    for h in (0.2, 0.1, 0.05):
        W1, _ = oracle.isomp_step(W0, h, tol=1e-15, maxit=200)
        ref = _rk4_reference(W0, h, 400)
        errs.append(np.abs(W1 - ref).max())
    # local error of a second-order one-step method is O(h^3)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.0 < r1 < 10.0 and 6.0 < r2 < 10.0, errs
    # and the sign of time is right: a reversed step is far off
    Wm, _ = oracle.isomp_step(W0, -0.1, tol=1e-15, maxit=200)
    assert np.abs(Wm - _rk4_reference(W0, 0.1, 400)).max() > 100 * errs[1]


def test_reversibility_and_invariants_over_steps():
    N, h, nsteps = 32, 0.01, 40
    W0 = vorticity_w0(N, seed=0)
    W, infos = oracle.isomp_run(W0, h, nsteps)
    assert all(i.converged for i in infos)
    assert max(i.iters for i in infos) <= 6
    # su(N) preserved
    assert np.abs(W + W.conj().T).max() < 1e-14
    assert abs(np.trace(W)) < 1e-13
    # isospectral: eigenvalues of the Hermitian matrix -iW are conserved
    ev0 = np.linalg.eigvalsh(-1j * W0)
    ev1 = np.linalg.eigvalsh(-1j * W)
    assert np.abs(ev1 - ev0).max() < 1e-12
    # Casimirs tr(W^k) conserved, relative to sum |lambda|^k
    c0, c1 = oracle.casimirs(W0, (2, 3, 4)), oracle.casimirs(W, (2, 3, 4))
    for k in (2, 3, 4):
        scale = np.sum(np.abs(ev0) ** k)
        assert abs(c1[k] - c0[k]) / scale < 1e-12, k
    # the flow moved
    assert np.abs(W - W0).max() > 1e-4
    # time reversal: stepping back with -h returns to W0
    Wb, _ = oracle.isomp_run(W, -h, nsteps)
    assert np.abs(Wb - W0).max() < 1e-12


def test_reuse_variant_close_to_fresh():
    N, h = 24, 0.01
    W0 = vorticity_w0(N, seed=2)
    Wf, _ = oracle.isomp_step(W0, h, final="fresh")
    Wr, _ = oracle.isomp_step(W0, h, final="reuse")
    assert np.linalg.norm(Wf - Wr) / np.linalg.norm(Wf) < 1e-12


def test_residual_history_contracts():
    N, h = 64, 0.01
    W0 = vorticity_w0(N, seed=0)
    _, info = oracle.isomp_step(W0, h, tol=1e-12)
    hist = info.history
    assert info.converged and 2 <= len(hist) <= 6
    for a, b in zip(hist, hist[1:]):
        assert b < 1e-2 * a


def test_fixed_point_does_not_depend_on_the_first_iterate():
    # Eq. 9 is a contraction for small h: from W_n or from the midpoint extrapolated
    # along the trajectory, W_n + (W_n - W_{n-1})/2, the same W_{n+1} (within tol),
    # the extrapolated start (an O(h^2) guess) in no more sweeps
    N, h = 48, 0.005
    W0 = vorticity_w0(N, seed=3)
    W1, _ = oracle.isomp_step(W0, h)
    plain, ip = oracle.isomp_step(W1, h)
    extra, ie = oracle.isomp_step(W1, h, Wt0=W1 + 0.5 * (W1 - W0))
    assert np.linalg.norm(extra - plain) / np.linalg.norm(plain) < 1e-14
    assert ie.converged and ie.iters <= ip.iters
    assert ie.history[0] < 1e-2 * ip.history[0]
    # a poor first iterate converges to the same point too
    far, iff = oracle.isomp_step(W1, h, Wt0=np.zeros_like(W1))
    assert iff.converged and np.linalg.norm(far - plain) / np.linalg.norm(plain) < 1e-14
