"""The oracle's Casimirs C_k = tr(W^k) (Sec. 2, Eq. 7) against the spectrum:
tr(W^k) = sum_j lambda_j^k for the eigenvalues of W (an eigensolver, not
repeated products)."""
import numpy as np
import pytest

import oracle
from paper_2206_05466_gb300.inputs import vorticity_w0


@pytest.mark.parametrize("N", [2, 5, 16, 40])
def test_casimirs_equal_power_sums_of_the_spectrum(N):
    W = vorticity_w0(N, seed=N)
    lam = 1j * np.linalg.eigvalsh(-1j * W)   # W = i H, H Hermitian: eigenvalues i mu
    got = oracle.casimirs(W, (2, 3, 4, 5))
    for k in (2, 3, 4, 5):
        want = np.sum(lam ** k)
        scale = np.sum(np.abs(lam) ** k)
        assert abs(got[k] - want) <= 1e-13 * scale, (k, got[k], want)
    # structure: even k real and of sign (-1)^(k/2), odd k purely imaginary
    assert abs(got[2].imag) <= 1e-14 * abs(got[2]) and got[2].real < 0
    assert abs(got[4].imag) <= 1e-14 * abs(got[4]) and got[4].real > 0
    assert abs(got[3].real) <= 1e-13 * np.sum(np.abs(lam) ** 3)
