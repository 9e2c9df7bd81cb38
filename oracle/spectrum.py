"""Oracle for the kinetic-energy spectrum E_l (Sec. 4; basis of Sec. 3.2).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path.

The paper plots the kinetic-energy spectrum against the spherical-harmonic
degree l without printing its formula.  It is taken here as
    E_l = sum_{|m| <= l} |omega_lm|^2 / (2 l (l+1)),   l = 1 .. N-1,   E_0 = 0,
with omega_lm the coefficients of W in the quantised basis (Eq. 10).  Because
P = Delta_N^{-1} W has coefficients -omega_lm / (l(l+1)) (Eq. 12), the E_l sum
to the Hamiltonian (1/2) tr(P W).

|omega_lm| does not depend on the sign of T^_lm, so each block is handled
with a library eigensolver and no sign rule: for diagonal m of W (lower,
W[i+m, i]) and -m (upper, W[i, i+m]), |omega_{l,+-m}| = |v_l^T w_{+-m}| with
v_l the unit eigenvector of -Delta^m (Eq. 13) for the eigenvalue l(l+1).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .zeitlin import laplacian_block


def energy_spectrum(W: np.ndarray) -> np.ndarray:
    """E_l, l = 0 .. N-1, of an N x N complex matrix W (see the module docstring)."""
    W = np.asarray(W, dtype=np.complex128)
    N = W.shape[0]
    E = np.zeros(N)
    for m in range(N):
        n = N - m
        a, b = laplacian_block(N, m)
        if n == 1:
            lam, V = a.copy(), np.ones((1, 1))
        else:
            lam, V = scipy.linalg.eigh_tridiagonal(a, b)
        l = np.arange(m, N)
        # Eq. 12: the block's eigenvalues are exactly l(l+1), l = m .. N-1, ascending
        assert np.allclose(lam, l * (l + 1.0), rtol=1e-9, atol=1e-9)
        lower = W[np.arange(m, N), np.arange(0, n)]
        e = np.abs(V.T @ lower) ** 2
        if m > 0:
            upper = W[np.arange(0, n), np.arange(m, N)]
            e += np.abs(V.T @ upper) ** 2
        E[m:] += e
    l = np.arange(1, N)
    E[1:] /= 2.0 * l * (l + 1.0)
    E[0] = 0.0
    return E
