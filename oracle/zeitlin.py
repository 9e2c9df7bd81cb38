"""Plain complex128 restatement of the IsoMP hot path (test infrastructure only).

Notation follows the paper: N matrix size, s = (N-1)/2, W vorticity matrix,
P stream matrix, h time step, W_n the state at time level n, Wt the implicit
midpoint matrix (W-tilde), Pt = Delta_N^{-1} Wt, k the fixed-point sweep.

Readings of the paper taken here (the CUDA path takes the same ones):
  * Sign of the blocks.  Eq. 13 prints a positive semidefinite
    tridiagonal matrix, while Eq. 12 gives Delta_N the eigenvalues
    -l(l+1).  The printed matrix is taken as T_m = -Delta^m: the block of
    Delta_N on diagonal m is -T_m.
  * Diagonal indexing.  Diagonal m (0 <= m <= N-1) of a matrix A is the
    vector A[i+m, i], i = 0..N-m-1 (Sec. 3.3); the super-diagonal -m,
    A[i, i+m], carries the same block T_m.
  * Singular block m = 0.  T_0 has the constant vector as null vector (the
    l = 0 mode).  The l = 0 mode is projected out: the right-hand side has its
    mean removed, the leading N-1 equations are solved with x[N-1] = 0, and
    the mean of x is removed.  This equals -T_0^+ W_0 and gives tr P = 0.
  * Third term of Eq. 9.  Read as Pt Wt Pt, the term obtained by
    expanding the first line of Eq. 8.
  * Stop rule.  Absolute Frobenius norm of Wt^{k+1} - Wt^k below tol, or
    maxit sweeps; Wt^0 = W_n.
  * Assembly of W_{n+1} ("fresh", default).  Pt, A = Pt Wt and B = A Pt are
    recomputed from the last iterate before the second line of Eq. 8 is
    applied (Sec. 3.1 counts two products for W_{n+1} as well).  "reuse"
    instead takes A and B of the last sweep.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

__all__ = [
    "laplacian_block",
    "laplacian_apply",
    "stream_solve",
    "isomp_step",
    "isomp_run",
    "casimirs",
    "StepInfo",
]


def laplacian_block(N: int, m: int):
    """Tridiagonal block T_m = -Delta^m of diagonal m (Sec. 3.2, Eq. 13).

    Returns (a, b): a[i] the diagonal entries, i = 0..N-m-1, and b[i] the
    symmetric off-diagonal entries T_m[i, i+1] = T_m[i+1, i], i = 0..N-m-2:
        a[i] = 2 (s (2i + 1 + m) - i (i + m)),             s = (N - 1)/2
        b[i] = -sqrt((i + m + 1)(N - 1 - i - m)) * sqrt((i + 1)(N - 1 - i)).
    The delta_{i-1} term of Eq. 13 is the same expression with i
    shifted by one, so the block is symmetric.
    """
    if not (0 <= m <= N - 1):
        raise ValueError("diagonal index out of range")
    n = N - m
    s = (N - 1) / 2.0
    i = np.arange(n, dtype=np.float64)
    a = 2.0 * (s * (2.0 * i + 1.0 + m) - i * (i + m))
    ii = np.arange(n - 1, dtype=np.float64)
    b = -np.sqrt((ii + m + 1.0) * (N - 1.0 - ii - m)) * np.sqrt((ii + 1.0) * (N - 1.0 - ii))
    return a, b


def _tridiag_matvec(a, b, v):
    """y = T v for the symmetric tridiagonal T with diagonal a, off-diagonal b."""
    y = a * v
    if v.shape[0] > 1:
        y[:-1] += b * v[1:]
        y[1:] += b * v[:-1]
    return y


def laplacian_apply(P: np.ndarray) -> np.ndarray:
    """W = Delta_N P for any complex N x N matrix P (Sec. 3.2-3.3).

    Delta_N acts on each diagonal separately (Eq. 14): on the
    sub-diagonal m and on the super-diagonal -m it is the block -T_m.
    """
    P = np.asarray(P, dtype=np.complex128)
    N = P.shape[0]
    W = np.zeros_like(P)
    for m in range(N):
        a, b = laplacian_block(N, m)
        i = np.arange(N - m)
        W[i + m, i] = -_tridiag_matvec(a, b, P[i + m, i])
        if m > 0:
            W[i, i + m] = -_tridiag_matvec(a, b, P[i, i + m])
    return W


def _solve_spd_tridiag(a, b, rhs):
    """x = T^{-1} rhs for symmetric positive definite tridiagonal T (library banded solve)."""
    n = a.shape[0]
    if n == 1:
        return rhs / a[0]
    ab = np.zeros((2, n), dtype=np.float64)
    ab[0, 1:] = b
    ab[1, :] = a
    return sla.solveh_banded(ab, rhs.astype(np.complex128), lower=False)


def stream_solve(W: np.ndarray) -> np.ndarray:
    """P = Delta_N^{-1} W for W in su(N) (Sec. 3.3, Eq. 14).

    For each diagonal m = 0..N-1 the lower diagonal P_m solves
    Delta^m P_m = W_m, i.e. P_m = -T_m^{-1} W_m; the l = 0 mode of the
    singular m = 0 block is projected out.  The upper triangle follows from
    skew-Hermitian symmetry, P[i, i+m] = -conj(P[i+m, i]).
    """
    W = np.asarray(W, dtype=np.complex128)
    N = W.shape[0]
    P = np.zeros_like(W)
    for m in range(N):
        a, b = laplacian_block(N, m)
        i = np.arange(N - m)
        rhs = W[i + m, i]
        if m == 0:
            rhs = rhs - rhs.mean()
            x = np.zeros(N, dtype=np.complex128)
            if N > 1:
                x[: N - 1] = _solve_spd_tridiag(a[: N - 1], b[: N - 2], rhs[: N - 1])
            x = x - x.mean()
        else:
            x = _solve_spd_tridiag(a, b, rhs)
        P[i + m, i] = -x
        if m > 0:
            P[i, i + m] = -np.conj(P[i + m, i])
    return P


@dataclass
class StepInfo:
    iters: int
    residual: float
    converged: bool
    history: list = field(default_factory=list)
    Wt: np.ndarray | None = None
    Pt: np.ndarray | None = None


def isomp_step(Wn: np.ndarray, h: float, tol: float = 1e-12, maxit: int = 50,
               final: str = "fresh", Wt0=None):
    """One isospectral-midpoint step W_n -> W_{n+1} (Sec. 2, Eqs. 8, 9).

    Fixed point (Eq. 9), with the two products of Sec. 3.1:
        Pt = Delta_N^{-1} Wt^k,  A = Pt Wt^k,  B = A Pt,
        Wt^{k+1} = W_n + h/2 (A - A^H) + h^2/4 B
    (Wt^k Pt = A^H because Pt and Wt are skew-Hermitian).  Then the second
    line of Eq. 8, W_{n+1} = Wt + h/2 (A - A^H) - h^2/4 B.
    Wt0 is the first iterate Wt^0 (the paper does not fix it; default W_n).
    Returns (W_{n+1}, StepInfo).
    """
    if final not in ("fresh", "reuse"):
        raise ValueError("final must be 'fresh' or 'reuse'")
    Wn = np.asarray(Wn, dtype=np.complex128)
    Wt = Wn.copy() if Wt0 is None else np.asarray(Wt0, dtype=np.complex128).copy()
    hist = []
    converged = False
    A = B = None
    iters = 0
    for k in range(maxit):
        Pt = stream_solve(Wt)
        A = Pt @ Wt
        B = A @ Pt
        Wnew = Wn + (h / 2.0) * (A - A.conj().T) + (h * h / 4.0) * B
        r = float(np.linalg.norm(Wnew - Wt))
        hist.append(r)
        Wt = Wnew
        iters = k + 1
        if r < tol:
            converged = True
            break
    if final == "fresh":
        Pt = stream_solve(Wt)
        A = Pt @ Wt
        B = A @ Pt
    Wnp1 = Wt + (h / 2.0) * (A - A.conj().T) - (h * h / 4.0) * B
    info = StepInfo(iters=iters, residual=hist[-1] if hist else 0.0,
                    converged=converged, history=hist, Wt=Wt, Pt=Pt)
    return Wnp1, info


def isomp_run(W0: np.ndarray, h: float, nsteps: int, tol: float = 1e-12,
              maxit: int = 50, final: str = "fresh", callback=None):
    """nsteps IsoMP steps from W0; returns (W, [StepInfo, ...])."""
    W = np.asarray(W0, dtype=np.complex128).copy()
    infos = []
    for n in range(nsteps):
        W, info = isomp_step(W, h, tol, maxit, final)
        info.Wt = info.Pt = None
        infos.append(info)
        if callback is not None:
            callback(n + 1, W, info)
    return W, infos


def casimirs(W: np.ndarray, ks=(2, 3, 4)):
    """Discrete Casimirs C_k(W) = tr(W^k) (Sec. 2, Eq. 7)."""
    W = np.asarray(W, dtype=np.complex128)
    out = {}
    M = np.eye(W.shape[0], dtype=np.complex128)
    for k in range(1, max(ks) + 1):
        M = M @ W
        if k in ks:
            out[k] = complex(np.trace(M))
    return out
