"""Oracle for the quantised spherical-harmonic basis (Sec. 3.2, Eqs. 10-12).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path.

* `wigner3j`: Wigner 3j symbols by Racah's closed formula, in exact integer
  and rational arithmetic (arguments doubled, so half-integers are exact);
  the square root is taken once at the end.
* `that_lm`: the complex basis matrix T^_lm of Eq. 11,
      (T^_lm)[i, j] = (-1)^(s - i) sqrt(2l+1) (s l s; -i m j),  s = (N-1)/2,
  with i, j in {-s, ..., s} and matrix row/column r = i + s, c = j + s (so
  T^_lm with m > 0 lies on the lower m-th diagonal, r - c = m).  The bracket
  [(N-1)/2] of Eq. 11 is read as s itself: s - i is an integer for every i.
* `that_lm_eig`: the same matrix from the eigenvector of the tridiagonal
  block -Delta^m with eigenvalue l(l+1) (Eqs. 12-13; SciPy's banded symmetric
  eigensolver), unit 2-norm, sign fixed by `SIGN_RULE`.
* `w_from_omega`, `omega_from_w`: Eq. 10 (W = sum i omega_lm T^_lm) and its
  inverse by orthonormality, omega_lm = -i tr(T^_lm^H W).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial, sqrt

import numpy as np
import scipy.linalg

from .zeitlin import laplacian_block


def wigner3j(j1: float, j2: float, j3: float, m1: float, m2: float, m3: float) -> float:
    """(j1 j2 j3; m1 m2 m3) by Racah's formula (exact up to the final sqrt)."""
    a = [int(round(2 * x)) for x in (j1, j2, j3, m1, m2, m3)]
    J1, J2, J3, M1, M2, M3 = a
    if M1 + M2 + M3 != 0:
        return 0.0
    if any((J + M) % 2 for J, M in ((J1, M1), (J2, M2), (J3, M3))) or any(abs(M) > J for J, M in
                                                                            ((J1, M1), (J2, M2), (J3, M3))):
        return 0.0
    if J3 > J1 + J2 or J3 < abs(J1 - J2) or (J1 + J2 + J3) % 2:
        return 0.0

    def f(x2):   # factorial of a doubled (integer-valued) argument
        assert x2 % 2 == 0 and x2 >= 0
        return factorial(x2 // 2)

    tri = Fraction(f(J1 + J2 - J3) * f(J1 - J2 + J3) * f(-J1 + J2 + J3), f(J1 + J2 + J3 + 2))
    pref = tri * f(J1 + M1) * f(J1 - M1) * f(J2 + M2) * f(J2 - M2) * f(J3 + M3) * f(J3 - M3)
    tmin = max(0, (J2 - J3 - M1) // 2, (J1 - J3 + M2) // 2)
    tmax = min((J1 + J2 - J3) // 2, (J1 - M1) // 2, (J2 + M2) // 2)
    ssum = Fraction(0)
    for t in range(tmin, tmax + 1):
        den = (factorial(t) * f(J3 - J2 + 2 * t + M1) * f(J3 - J1 + 2 * t - M2) * f(J1 + J2 - J3 - 2 * t) *
               f(J1 - 2 * t - M1) * f(J2 - 2 * t + M2))
        ssum += Fraction((-1) ** t, den)
    e = J1 - J2 - M3   # (-1)^(j1 - j2 - m3), an integer exponent once halved
    assert e % 2 == 0
    sign = -1.0 if (e // 2) % 2 else 1.0
    val = ssum * ssum * pref   # square of the magnitude, exact
    mag = sqrt(float(val))
    return sign * (mag if ssum >= 0 else -mag)


def that_lm(N: int, l: int, m: int) -> np.ndarray:
    """T^_lm of Eq. 11 (real entries, N x N)."""
    s = (N - 1) / 2
    T = np.zeros((N, N))
    for r in range(N):
        i = r - s
        j = i - m   # the 3j symbol vanishes unless -i + m + j = 0
        c = int(round(j + s))
        if 0 <= c < N:
            e = int(round(s - i))
            T[r, c] = (-1) ** e * sqrt(2 * l + 1) * wigner3j(s, l, s, -i, m, j)
    return T


def SIGN_RULE(N: int, l: int, m: int) -> int:
    """Sign of the last entry (position N - m - 1) of the m-th diagonal of T^_lm, m >= 0.

    There i = s and j = s - m, so Eq. 11 reads sqrt(2l+1) (s l s; -s m s-m)
    times (-1)^(s-i) = 1.  Reflecting all m's, (j1 j2 j3; m1 m2 m3) =
    (-1)^(j1+j2+j3) (j1 j2 j3; -m1 -m2 -m3), gives (-1)^(2s+l) (s l s; s -m m-s),
    whose first column is stretched (m1 = j1): Racah's sum has the single
    term t = 0 > 0, so its sign is (-1)^(j1-j2-m3) = (-1)^(2s-l-m).  Together:
    (-1)^(4s-m) = (-1)^m, since 4s = 2(N-1) is even.
    """
    return -1 if m % 2 else 1


def end_recurrence_sign(d, e, lam, sign_last, j):
    """Sign at position j of the solution of (T - lam I) y = 0 (T tridiagonal: diagonal d,
    off-diagonal e, all e < 0) with y[n-1] = sign_last, by the backward three-term
    recurrence (rescaled against overflow)."""
    n = len(d)
    y1, y0 = float(sign_last), 0.0   # y[i], y[i+1]
    for i in range(n - 1, j, -1):
        # row i: e[i-1] y[i-1] + (d[i] - lam) y[i] + e[i] y[i+1] = 0
        nxt = -((d[i] - lam) * y1 + (e[i] * y0 if i + 1 < n else 0.0)) / e[i - 1]
        y0, y1 = y1, nxt
        big = max(abs(y0), abs(y1))
        if big > 1e100:
            y0, y1 = y0 / big, y1 / big
    return float(np.sign(y1))


def that_lm_eig(N: int, l: int, m: int) -> np.ndarray:
    """T^_lm from the eigenvector of the block -Delta^m for the eigenvalue l(l+1), m >= 0."""
    assert 0 <= m <= l < N
    n = N - m
    d, e = laplacian_block(N, m)   # -Delta^m: diagonal, off-diagonal; eigenvalues l(l+1), l = m .. N-1
    if n == 1:
        lam, vec = np.array([d[0]]), np.ones((1, 1))
    else:
        lam, vec = scipy.linalg.eigh_tridiagonal(d, e)
    k = int(np.argmin(np.abs(lam - l * (l + 1))))
    v = vec[:, k] / np.linalg.norm(vec[:, k])
    # The end entries can be far below the eigensolver's absolute accuracy (and
    # interior entries can vanish: the blocks are persymmetric), so the sign is
    # fixed at the largest entry: the three-term recurrence of (-Delta^m -
    # l(l+1) I) y = 0 run backwards from y[n-1] = (-1)^m (the sign the
    # stretched 3j symbol gives the last entry) grows from that end towards
    # the bulk, and its sign at the largest entry of v is that of T^_lm there.
    jmax = int(np.argmax(np.abs(v)))
    if end_recurrence_sign(d, e, l * (l + 1), SIGN_RULE(N, l, m), jmax) != np.sign(v[jmax]):
        v = -v
    out = np.zeros((N, N))
    out[np.arange(m, N), np.arange(0, n)] = v
    return out


def omega_index(l: int, m: int) -> int:
    """Position of omega_lm in a flat array over l = 0.., m = -l..l."""
    return l * l + l + m


def w_from_omega(N: int, omega: np.ndarray, lmax: int) -> np.ndarray:
    """W = sum_{l <= lmax} sum_m i omega_lm T^_lm (Eq. 10), T^_{l,-m} = (-1)^m T^_lm^T for m > 0."""
    W = np.zeros((N, N), dtype=np.complex128)
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            T = that_lm(N, l, m)
            W += 1j * omega[omega_index(l, m)] * T
            if m > 0:
                W += 1j * omega[omega_index(l, -m)] * ((-1) ** m) * T.T
    return W


def omega_from_w(N: int, W: np.ndarray, lmax: int, route: str = "3j") -> np.ndarray:
    """omega_lm = -i tr(T^_lm^H W) (orthonormal basis), l <= lmax.

    route "3j" builds T^_lm from Eq. 11 (exact 3j symbols, slow beyond N ~ 100);
    route "eig" from the eigenvectors of the blocks with the sign rule (Sec. 3.2).
    """
    make = {"3j": that_lm, "eig": that_lm_eig}[route]
    out = np.zeros((lmax + 1) ** 2, dtype=np.complex128)
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            T = make(N, l, m)
            out[omega_index(l, m)] = -1j * np.sum(T * W)   # T real: tr(T^T W) = sum T_rc W_rc
            if m > 0:
                out[omega_index(l, -m)] = -1j * ((-1) ** m) * np.sum(T.T * W)
    return out
