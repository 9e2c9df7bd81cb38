"""Pins of the oracle's Laplacian blocks and stream solve (CPU only).

The pins come from outside the oracle: the closed-form spectrum of Eq.
12, hand-worked blocks of Eq. 13, and the textbook spin-Casimir
construction of Hoppe's Laplacian (tests/_spin.py), inverted densely.
"""
import os

import numpy as np
import pytest

import oracle
from tests import _spin

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "laplacian_blocks_small.txt")


def _read_golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, diag, off, eig = [p.strip() for p in line.split("|")]
            N, m = (int(x) for x in head.split())
            rows.append((N, m, [float(x) for x in diag.split()],
                         [float(x) for x in off.split()], [float(x) for x in eig.split()]))
    return rows


def test_blocks_match_hand_worked_golden():
    rows = _read_golden()
    assert len(rows) >= 6
    for N, m, diag, off, eig in rows:
        a, b = oracle.laplacian_block(N, m)
        np.testing.assert_allclose(a, diag, rtol=0, atol=1e-14)
        np.testing.assert_allclose(b, off, rtol=0, atol=1e-14)
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        np.testing.assert_allclose(np.linalg.eigvalsh(T), eig, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 8, 13, 32])
def test_block_spectrum_is_l_l_plus_1(N):
    # Eq. 12 restricted to diagonal m: eigenvalues l(l+1), l = m..N-1.
    for m in range(N):
        a, b = oracle.laplacian_block(N, m)
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        ev = np.linalg.eigvalsh(T)
        l = np.arange(m, N, dtype=np.float64)
        np.testing.assert_allclose(ev, l * (l + 1), rtol=1e-13, atol=1e-11)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 8])
def test_dense_spectrum_of_laplacian_apply(N):
    # Full operator: eigenvalues -l(l+1), multiplicity 2l+1, l = 0..N-1.
    L = np.zeros((N * N, N * N))
    for idx in range(N * N):
        E = np.zeros(N * N)
        E[idx] = 1.0
        L[:, idx] = oracle.laplacian_apply(E.reshape(N, N)).real.reshape(-1)
    np.testing.assert_allclose(L, L.T, atol=1e-12)
    ev = np.sort(np.linalg.eigvalsh(L))
    want = np.sort(np.concatenate([[-l * (l + 1.0)] * (2 * l + 1) for l in range(N)]))
    np.testing.assert_allclose(ev, want, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 9, 16])
def test_laplacian_equals_spin_casimir(N):
    # Every block, both sub- and super-diagonals, and the sign: the oracle's
    # Delta_N must equal -sum_a [S_a, [S_a, .]] on arbitrary complex matrices.
    rng = np.random.default_rng(N)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    got = oracle.laplacian_apply(X)
    want = _spin.casimir_laplacian(X)
    scale = max(1.0, np.abs(want).max())
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * scale * N)


@pytest.mark.parametrize("N", [2, 3, 4, 6, 9, 12])
def test_stream_solve_equals_dense_pseudo_inverse(N):
    Linv = _spin.dense_pseudo_inverse(N)
    for seed in range(3):
        W = _spin.random_su(N, seed)
        P = oracle.stream_solve(W)
        want = (Linv @ W.reshape(-1)).reshape(N, N)
        np.testing.assert_allclose(P, want, rtol=0, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("N", [33, 64, 130])
def test_stream_solve_roundtrip_and_structure(N):
    from paper_2206_05466_gb300.inputs import vorticity_w0

    W = vorticity_w0(N, seed=1)
    P = oracle.stream_solve(W)
    # Delta_N P = W, with Delta_N built independently from spin matrices.
    back = _spin.casimir_laplacian(P)
    np.testing.assert_allclose(back, W, rtol=0, atol=1e-12 * np.abs(W).max())
    # P in su(N): skew-Hermitian and traceless (Sec. 3.3).
    assert np.abs(P + P.conj().T).max() == 0.0
    assert abs(np.trace(P)) < 1e-14 * np.abs(P).max() * N


def test_stream_solve_eigenmodes():
    # W in the l-eigenspace of Delta_N gives P = -W / (l(l+1)) (Eq. 12).
    N = 11
    S1, S2, S3 = _spin.spin_matrices(N)
    s = (N - 1) / 2
    W1 = 1j * (0.3 * S1 - 0.7 * S2 + 0.2 * S3)               # l = 1
    W2 = 1j * (S3 @ S3 - s * (s + 1) / 3 * np.eye(N))        # l = 2
    np.testing.assert_allclose(oracle.stream_solve(W1), -W1 / 2, atol=1e-14)
    np.testing.assert_allclose(oracle.stream_solve(W2), -W2 / 6, atol=1e-13)


def test_n1_is_zero():
    assert oracle.stream_solve(np.zeros((1, 1), complex)).tolist() == [[0j]]
    assert oracle.laplacian_apply(np.ones((1, 1), complex)).tolist() == [[0j]]


def test_m0_projection_removes_trace():
    # A right-hand side with a trace: the l = 0 part is discarded, the result
    # is the minimum-norm least-squares solution (pseudo-inverse).
    N = 7
    rng = np.random.default_rng(5)
    W = _spin.random_su(N, 2) + 0.3j * np.eye(N)
    P = oracle.stream_solve(W)
    want = (_spin.dense_pseudo_inverse(N) @ W.reshape(-1)).reshape(N, N)
    np.testing.assert_allclose(P, want, atol=1e-13)
    assert abs(np.trace(P)) < 1e-14
    del rng
