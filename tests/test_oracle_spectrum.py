"""Pins of the kinetic-energy spectrum oracle (Sec. 4 with the basis of Sec. 3.2).

Facts that do not come from the spectrum oracle: single basis matrices built
by the Wigner 3j route (Eq. 11), the brute-force sum over known coefficients,
Parseval's identity for an orthonormal basis, and the Hamiltonian (1/2) tr(P W)
with the separately pinned stream solve.
"""
import numpy as np
import pytest

import oracle
from oracle import basis
from oracle.spectrum import energy_spectrum
from paper_2206_05466_gb300.inputs import paper_omega, vorticity_w0


@pytest.mark.parametrize("N,l,m", [(2, 1, 0), (2, 1, 1), (3, 2, -2), (5, 3, 1), (5, 3, -1), (8, 7, 0),
                                   (8, 4, -3), (9, 8, 8)])
def test_single_mode(N, l, m):
    c = 0.7 - 1.3j
    if m >= 0:
        T = basis.that_lm(N, l, m)
    else:
        T = (-1) ** (-m) * basis.that_lm(N, l, -m).T
    E = energy_spectrum(1j * c * T)
    want = np.zeros(N)
    want[l] = abs(c) ** 2 / (2 * l * (l + 1))
    assert np.abs(E - want).max() < 1e-14


@pytest.mark.parametrize("N", [2, 3, 6, 9])
def test_known_coefficients(N):
    om = paper_omega(N - 1, lmin=1, seed=N)
    W = basis.w_from_omega(N, om, N - 1)
    E = energy_spectrum(W)
    for l in range(1, N):
        want = sum(abs(om[l * l + l + m]) ** 2 for m in range(-l, l + 1)) / (2 * l * (l + 1))
        assert abs(E[l] - want) < 1e-13 * max(1.0, want), l
    assert E[0] == 0.0


@pytest.mark.parametrize("N", [4, 17, 64])
def test_parseval_and_hamiltonian(N):
    W = vorticity_w0(N, seed=5)
    E = energy_spectrum(W)
    l = np.arange(N)
    # orthonormal basis: sum_lm |omega_lm|^2 = ||W||_F^2 (omega_00 = 0 in su(N))
    fro2 = np.sum(W.real ** 2 + W.imag ** 2)
    assert abs(np.sum(2 * l * (l + 1) * E) - fro2) < 1e-12 * fro2
    # the E_l sum to the Hamiltonian (1/2) tr(P W), P = Delta_N^{-1} W
    P = oracle.stream_solve(W)
    H = 0.5 * np.trace(P @ W)
    assert abs(H.imag) < 1e-12 * abs(H.real)
    assert abs(E.sum() - H.real) < 1e-12 * abs(H.real)
    assert (E >= 0).all()


@pytest.mark.parametrize("N,L", [(2, 1), (5, 4), (33, 8), (128, 6), (129, 12)])
def test_extended_low_modes_equal_the_eigensolver_route(N, L):
    from oracle.spectrum import energy_spectrum_low
    W = vorticity_w0(N, seed=9)
    full = energy_spectrum(W)
    low = energy_spectrum_low(W, L).astype(np.float64)
    assert low[0] == 0.0
    assert np.abs(low[1:] - full[1:L + 1]).max() <= 1e-12 * full[1:L + 1].max()


def test_extended_low_modes_known_coefficients():
    from oracle.spectrum import energy_spectrum_low
    N = 9
    om = paper_omega(N - 1, lmin=1, seed=3)
    E = energy_spectrum_low(basis.w_from_omega(N, om, N - 1), 5).astype(np.float64)
    for l in range(1, 6):
        want = sum(abs(om[l * l + l + m]) ** 2 for m in range(-l, l + 1)) / (2 * l * (l + 1))
        assert abs(E[l] - want) < 1e-14 * want


@pytest.mark.parametrize("N", [2, 5, 8, 11])
def test_reflection_parity_of_the_3j_basis(N):
    # the half-vector routes rely on x_{n-1-i} = (-1)^(l-m) x_i along the diagonal (Eq. 11)
    for l in range(N):
        for m in range(l + 1):
            v = np.diag(basis.that_lm(N, l, m), -m)
            assert np.abs(v[::-1] - (-1) ** (l - m) * v).max() < 1e-14, (l, m)


def test_restricting_to_the_occupied_diagonals_changes_nothing():
    # a matrix with content on a few diagonals only: visiting just those blocks
    # gives the same spectrum as visiting all of them
    N = 40
    rng = np.random.default_rng(3)
    W = np.zeros((N, N), complex)
    for m in (0, 2, 17, 39):
        v = rng.standard_normal(N - m) + 1j * rng.standard_normal(N - m)
        W[np.arange(m, N), np.arange(0, N - m)] = v
        W[np.arange(0, N - m), np.arange(m, N)] = -np.conj(v)
    W[np.diag_indices(N)] = 1j * W[np.diag_indices(N)].imag
    assert np.array_equal(energy_spectrum(W, diagonals=[0, 2, 17, 39]), energy_spectrum(W))
    with pytest.raises(AssertionError):
        energy_spectrum(W, diagonals=[0, 2])
