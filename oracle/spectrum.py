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


def energy_spectrum(W: np.ndarray, diagonals=None) -> np.ndarray:
    """E_l, l = 0 .. N-1, of an N x N complex matrix W (see the module docstring).

    `diagonals`: if given, W must vanish off the diagonals +-m for m in it (checked),
    and only those blocks are visited (the others contribute nothing).
    """
    W = np.asarray(W, dtype=np.complex128)
    N = W.shape[0]
    E = np.zeros(N)
    ms = range(N)
    if diagonals is not None:
        ms = sorted(set(int(m) for m in diagonals))
        r, c = np.indices((N, N))
        assert not np.any(W[~np.isin(np.abs(r - c), ms)]), "W has content on other diagonals"
    for m in ms:
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


def energy_spectrum_low(W: np.ndarray, L: int) -> np.ndarray:
    """E_l for l = 0 .. L in extended precision (np.longdouble), for checks at large N.

    The library eigensolver above works on blocks rounded to double, and for
    the lowest l at large N (a_i ~ N^2 against l(l+1)) its eigenvectors carry
    relative errors up to about N^2 eps (1e-11 at N = 4096).  Here each
    eigenvector comes from the rows of Eq. 13 at the exact eigenvalue l(l+1)
    (Eq. 12), x_{i+1} = ((l(l+1) - a_i) x_i - b_{i-1} x_{i-1}) / b_i from x_0 = 1,
    in extended precision with the block entries evaluated in it, up to the
    centre of the diagonal; the rest follows from the reflection symmetry of
    the 3j symbols of Eq. 11, x_{n-1-i} = (-1)^(l-m) x_i.  The recurrence runs
    in its stable direction there (growing from the end of the diagonal into
    the central oscillatory range).  E_0 = 0.
    """
    LD = np.longdouble
    W = np.asarray(W, dtype=np.complex128)
    N = W.shape[0]
    L = min(int(L), N - 1)
    E = np.zeros(L + 1, dtype=LD)
    s = LD(N - 1) / 2
    for m in range(L + 1):
        n = N - m
        i = np.arange(n, dtype=LD)
        a = 2 * (s * (2 * i + 1 + m) - i * (i + m))                      # Eq. 13, extended precision
        ii = i[:-1]
        b = -np.sqrt((ii + m + 1) * (N - 1 - ii - m)) * np.sqrt((ii + 1) * (N - 1 - ii))
        ls = np.arange(m, L + 1)
        lam = (ls * (ls + 1)).astype(LD)
        half = (n + 1) // 2
        X = np.zeros((n, len(ls)), dtype=LD)
        X[0] = 1
        for k in range(half - 1):
            prev = X[k - 1] * b[k - 1] if k > 0 else 0
            X[k + 1] = ((lam - a[k]) * X[k] - prev) / b[k]
        sign = np.where((ls - m) % 2, -1, 1).astype(LD)
        for k in range(half, n):
            X[k] = sign * X[n - 1 - k]
        nrm = (X * X).sum(axis=0)
        diags = [W[np.arange(m, N), np.arange(0, n)]]
        if m > 0:
            diags.append(W[np.arange(0, n), np.arange(m, N)])
        for w in diags:
            re = X.T @ w.real.astype(LD)
            im = X.T @ w.imag.astype(LD)
            E[m:] += (re * re + im * im) / nrm
    l = np.arange(1, L + 1).astype(LD)
    E[1:] /= 2 * l * (l + 1)
    E[0] = 0
    return E
