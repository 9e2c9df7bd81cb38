"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds only input generation; none of the IsoMP method's arithmetic
(Laplacian, stream solve, fixed-point sweep) lives here.

The paper's own initial condition (random spherical-harmonic coefficients
omega_lm for 2 <= l <= 20, Sec. 4) needs the quantised basis of Sec. 3.2. The
stand-in used everywhere in this project is a seeded vorticity matrix with the
same structure the method relies on: W0 is traceless and skew-Hermitian
(W0 in su(N), Eq. 6) and normalised in the spectral norm, as the
paper states its initial vorticity always is (Sec. 2, after Eq. 9).

Recipe (fixed, in this order):
  1. g = a + i b, a and b (N x N) standard normal draws from
     numpy.random.default_rng(seed): all of a first (row-major), then all of b;
  2. g[j, k] *= (1 + |j - k|) ** (-decay)      (decay = 2 by default);
  3. H = (g + g^H) / 2                          (Hermitian, exactly);
  4. H /= ||H||_2                               (largest |eigenvalue|);
  5. W0 = i (H - tr(H)/N I)                     (traceless, skew-Hermitian).
"""
from __future__ import annotations

import numpy as np

__all__ = ["vorticity_w0", "ensemble_sizes", "serving_jobs"]


def _spectral_norm_hermitian(H: np.ndarray) -> float:
    """Largest |eigenvalue| of a Hermitian matrix (its spectral norm)."""
    n = H.shape[0]
    if n <= 512:
        ev = np.linalg.eigvalsh(H)
        return float(max(abs(ev[0]), abs(ev[-1])))
    import scipy.linalg as sla

    lo = sla.eigvalsh(H, subset_by_index=[0, 0], driver="evr")[0]
    hi = sla.eigvalsh(H, subset_by_index=[n - 1, n - 1], driver="evr")[0]
    return float(max(abs(lo), abs(hi)))


def vorticity_w0(N: int, seed: int = 0, decay: float = 2.0) -> np.ndarray:
    """Seeded initial vorticity matrix W0 (complex128, N x N, C-contiguous)."""
    if N < 1:
        raise ValueError("N must be >= 1")
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((N, N))
    b = rng.standard_normal((N, N))
    g = a + 1j * b
    j = np.arange(N)
    g *= (1.0 + np.abs(j[:, None] - j[None, :])) ** (-float(decay))
    H = (g + g.conj().T) / 2.0
    nrm = _spectral_norm_hermitian(H)
    if nrm > 0.0:
        H = H / nrm
    H = H - (np.trace(H).real / N) * np.eye(N)
    W0 = 1j * H
    return np.ascontiguousarray(W0, dtype=np.complex128)


def ensemble_sizes(count: int = 256, choices=(128, 256, 384, 512), seed: int = 0) -> list[int]:
    """Matrix sizes of an ensemble: N drawn uniformly from `choices`."""
    rng = np.random.default_rng(seed)
    return [int(choices[i]) for i in rng.integers(0, len(choices), size=count)]


def serving_jobs(duration_s: float, rate_per_s: float = 50.0,
                 sizes=(256, 512, 1024, 2048), weights=(0.4, 0.3, 0.2, 0.1),
                 steps_range=(200, 2000), seed: int = 0):
    """Seeded Poisson job stream: list of (arrival_s, N, nsteps, w0_seed)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        N = int(rng.choice(sizes, p=np.asarray(weights) / np.sum(weights)))
        nsteps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        jobs.append((t, N, nsteps, len(jobs)))
    return jobs


def paper_omega(lmax: int = 20, lmin: int = 2, seed: int = 0):
    """Seeded spherical-harmonic coefficients of the paper's initial condition
    (Sec. 4: random omega_lm for 2 <= l <= 20): complex Gaussian omega_lm for
    m > 0 and real Gaussian omega_l0, with omega_{l,-m} = (-1)^m conj(omega_lm)
    (so that the vorticity is real / the matrix skew-Hermitian), stored flat at
    l*l + l + m over l <= lmax.  Random numbers only; the assembly of W from
    them is the library's (zeitlin_w_from_omega)."""
    import numpy as np

    rng = np.random.default_rng(seed)
    om = np.zeros((lmax + 1) ** 2, dtype=np.complex128)
    for l in range(lmin, lmax + 1):
        om[l * l + l] = rng.standard_normal()
        for m in range(1, l + 1):
            z = rng.standard_normal() + 1j * rng.standard_normal()
            om[l * l + l + m] = z
            om[l * l + l - m] = (-1) ** m * np.conj(z)
    return om
