"""Independent constructions used to pin the oracle (no code shared with oracle/).

Hoppe's discrete Laplacian on u(N) is the (negated) quadratic Casimir of the
adjoint action of a spin-s representation of su(2), s = (N-1)/2:
    Delta_N X = - sum_a [S_a, [S_a, X]],
whose eigenvalues are -l(l+1), l = 0..N-1, each 2l+1 times (the decomposition
of spin s (x) spin s into spins l = 0..2s).  The spin matrices below are the
textbook angular-momentum matrices in the basis |s, mu>, mu = s, s-1, ..., -s.
"""
from __future__ import annotations

import numpy as np


def spin_matrices(N: int):
    s = (N - 1) / 2.0
    mu = s - np.arange(N)
    S3 = np.diag(mu).astype(np.complex128)
    Sp = np.zeros((N, N), dtype=np.complex128)
    for i in range(1, N):
        # S_+ |mu_i> = sqrt(s(s+1) - mu_i(mu_i+1)) |mu_i + 1>, and mu_i + 1 = mu_{i-1}
        Sp[i - 1, i] = np.sqrt(s * (s + 1) - mu[i] * (mu[i] + 1))
    Sm = Sp.conj().T
    S1 = (Sp + Sm) / 2.0
    S2 = (Sp - Sm) / 2.0j
    return S1, S2, S3


def casimir_laplacian(X: np.ndarray) -> np.ndarray:
    """-sum_a [S_a, [S_a, X]] by explicit commutators."""
    N = X.shape[0]
    out = np.zeros((N, N), dtype=np.complex128)
    for S in spin_matrices(N):
        C = S @ X - X @ S
        out -= S @ C - C @ S
    return out


def dense_laplacian(N: int) -> np.ndarray:
    """N^2 x N^2 matrix of X -> -sum_a [S_a,[S_a,X]] on row-major vec(X)."""
    L = np.zeros((N * N, N * N), dtype=np.complex128)
    for idx in range(N * N):
        E = np.zeros(N * N, dtype=np.complex128)
        E[idx] = 1.0
        L[:, idx] = casimir_laplacian(E.reshape(N, N)).reshape(-1)
    return L


def dense_pseudo_inverse(N: int) -> np.ndarray:
    """Moore-Penrose inverse of the dense Laplacian via its eigendecomposition.

    The Laplacian is real symmetric in this basis; its only zero eigenvalue
    (the identity matrix, l = 0) is dropped explicitly, every other eigenvalue
    is <= -2.
    """
    L = dense_laplacian(N).real
    ev, V = np.linalg.eigh(L)
    inv = np.where(np.abs(ev) > 0.5, 1.0 / np.where(np.abs(ev) > 0.5, ev, 1.0), 0.0)
    return (V * inv) @ V.T


def random_su(N: int, seed: int) -> np.ndarray:
    """Random traceless skew-Hermitian matrix (no structure beyond su(N))."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    H = (g + g.conj().T) / 2
    H -= np.trace(H).real / N * np.eye(N)
    return 1j * H
