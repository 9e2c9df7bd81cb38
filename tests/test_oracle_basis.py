"""Pins of the quantised-basis oracle (Sec. 3.2, Eqs. 10-12).

Facts that do not come from the oracle: tabulated Wigner 3j values and their
orthogonality relation, the Laplacian eigen-relation (with the Laplacian
pinned separately against the spin-Casimir superoperator), orthonormality,
the adjoint relation between m and -m, su(N) membership under the reality
condition of the coefficients, and agreement of two independent routes to the
basis (3j symbols and a LAPACK tridiagonal eigensolver).
"""
from math import sqrt

import numpy as np
import pytest

import oracle
from oracle import basis


@pytest.mark.parametrize("args,want", [
    ((1, 1, 0, 0, 0, 0), -1 / sqrt(3)),
    ((1, 1, 0, 1, -1, 0), 1 / sqrt(3)),
    ((0.5, 0.5, 0, 0.5, -0.5, 0), 1 / sqrt(2)),
    ((1, 1, 2, 0, 0, 0), sqrt(2 / 15)),
    ((2, 2, 2, 0, 0, 0), -sqrt(2 / 35)),
    ((1, 1, 1, 1, 0, -1), -1 / sqrt(6)),
    ((1.5, 1.5, 0, 0.5, -0.5, 0), -0.5),
    ((2, 1, 1, 0, 0, 0), sqrt(2 / 15)),
])
def test_wigner3j_table_values(args, want):
    assert abs(basis.wigner3j(*args) - want) < 1e-14


@pytest.mark.parametrize("j1,j2", [(1, 1), (1.5, 1), (2, 1.5), (2.5, 2)])
def test_wigner3j_orthogonality(j1, j2):
    js = np.arange(abs(j1 - j2), j1 + j2 + 1)
    m1s = np.arange(-j1, j1 + 1)
    m2s = np.arange(-j2, j2 + 1)
    for j3 in js:
        for j3p in js:
            for m3 in np.arange(-min(j3, j3p), min(j3, j3p) + 1):
                s = sum(basis.wigner3j(j1, j2, j3, a, b, m3) * basis.wigner3j(j1, j2, j3p, a, b, m3)
                        for a in m1s for b in m2s)
                assert abs((2 * j3 + 1) * s - (1.0 if j3 == j3p else 0.0)) < 1e-13


@pytest.mark.parametrize("N", [2, 3, 6, 9])
def test_basis_is_the_laplacian_eigenbasis_and_orthonormal(N):
    Ts = {}
    for l in range(N):
        for m in range(-l, l + 1):
            T = basis.that_lm(N, l, m)
            lap = oracle.laplacian_apply(T.astype(np.complex128))
            assert np.abs(lap + l * (l + 1) * T).max() <= 1e-12 * max(1, l * (l + 1)), (l, m)
            Ts[(l, m)] = T
    keys = list(Ts)
    G = np.array([[np.sum(Ts[a] * Ts[b]) for b in keys] for a in keys])
    assert np.abs(G - np.eye(len(keys))).max() < 1e-13


@pytest.mark.parametrize("N", [3, 6, 9])
def test_adjoint_relation_between_m_and_minus_m(N):
    for l in range(N):
        for m in range(1, l + 1):
            assert np.abs(basis.that_lm(N, l, -m) - (-1) ** m * basis.that_lm(N, l, m).T).max() < 1e-14


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 12])
def test_eigenvector_route_with_sign_rule_equals_3j_route(N):
    for l in range(N):
        for m in range(0, l + 1):
            assert np.abs(basis.that_lm(N, l, m) - basis.that_lm_eig(N, l, m)).max() < 1e-13, (l, m)


def _real_omega(lmax, seed, lmin=0):
    rng = np.random.default_rng(seed)
    om = np.zeros((lmax + 1) ** 2, dtype=np.complex128)
    for l in range(lmin, lmax + 1):
        om[basis.omega_index(l, 0)] = rng.standard_normal()
        for m in range(1, l + 1):
            z = rng.standard_normal() + 1j * rng.standard_normal()
            om[basis.omega_index(l, m)] = z
            om[basis.omega_index(l, -m)] = (-1) ** m * np.conj(z)
    return om


@pytest.mark.parametrize("N,lmax", [(4, 3), (7, 5), (10, 9)])
def test_w_from_omega_is_in_su_n_and_round_trips(N, lmax):
    om = _real_omega(lmax, seed=N, lmin=1)
    W = basis.w_from_omega(N, om, lmax)
    assert np.abs(W + W.conj().T).max() < 1e-13
    assert abs(np.trace(W)) < 1e-13
    back = basis.omega_from_w(N, W, lmax)
    assert np.abs(back - om).max() < 1e-13
    assert np.abs(basis.omega_from_w(N, W, lmax, route="eig") - om).max() < 1e-13


@pytest.mark.parametrize("N,pairs", [(64, [(50, 40), (63, 63), (40, 1), (63, 0), (30, 29), (17, 9)]),
                                     (129, [(128, 100), (90, 90), (20, 3), (127, 64)])])
def test_eigenvector_route_at_larger_n_where_the_ends_are_tiny(N, pairs):
    for l, m in pairs:
        assert np.abs(basis.that_lm(N, l, m) - basis.that_lm_eig(N, l, m)).max() < 1e-13, (l, m)
