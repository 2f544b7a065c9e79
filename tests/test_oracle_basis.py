"""Pins of the oracle's 1-D operator tables against closed forms and library routines."""
import math

import numpy as np
import pytest

from oracle import basis


def test_lgl_closed_form_N5():
    # N=5 LGL nodes: +-1, +-sqrt(1/3 -+ 2 sqrt(7)/21); weights 1/15, (14 -+ sqrt 7)/30
    x, w = basis.lgl_nodes_weights(5)
    a = math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21)
    b = math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21)
    np.testing.assert_allclose(x, [-1, -b, -a, a, b, 1], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [1 / 15, (14 - math.sqrt(7)) / 30, (14 + math.sqrt(7)) / 30,
                                   (14 + math.sqrt(7)) / 30, (14 - math.sqrt(7)) / 30, 1 / 15], rtol=1e-14)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 9])
def test_lgl_quadrature_exactness(N):
    x, w = basis.lgl_nodes_weights(N)
    for k in range(2 * N):  # exact for degree <= 2N-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13
    # interior nodes are roots of L_N'
    if N > 1:
        _, dL = basis.legendre(N, x[1:-1])
        assert np.abs(dL).max() < 1e-12


@pytest.mark.parametrize("N", [2, 4, 5, 7])
def test_diff_matrix_exact_on_polynomials(N):
    x, _ = basis.lgl_nodes_weights(N)
    D = basis.diff_matrix(N, x)
    for k in range(N + 1):
        d = k * x ** (k - 1) if k else np.zeros_like(x)
        np.testing.assert_allclose(D @ x ** k, d, atol=1e-12)


def test_vandermonde_matches_numpy_legendre():
    x, _ = basis.lgl_nodes_weights(6)
    V = basis.vandermonde(6, x)
    for j in range(7):
        c = np.zeros(j + 1)
        c[j] = 1
        np.testing.assert_allclose(V[:, j], np.polynomial.legendre.legval(x, c), atol=1e-14)


def test_filter_values_and_action():
    s = basis.filter_sigma(5)
    assert s[:4].tolist() == [1.0, 1.0, 1.0, 1.0]
    assert abs(s[4] - math.exp(-36 * 0.8 ** 100)) < 1e-18 and abs(1 - s[4] - 7.33e-9) < 1e-11
    assert abs(s[5] - math.exp(-36)) < 1e-30
    x, _ = basis.lgl_nodes_weights(5)
    F = basis.filter_matrix(5, x)
    for k in range(4):  # degree <= N-2 untouched
        np.testing.assert_allclose(F @ x ** k, x ** k, atol=1e-14)
    L5 = np.polynomial.legendre.legval(x, [0, 0, 0, 0, 0, 1])
    np.testing.assert_allclose(F @ L5, math.exp(-36) * L5, atol=1e-14)


def test_tci_lowpass():
    x, _ = basis.lgl_nodes_weights(5)
    Pi = basis.tci_lowpass_matrix(5, x, 3)
    for k in range(3):
        np.testing.assert_allclose(Pi @ x ** k, x ** k, atol=1e-14)
    for j in (3, 4, 5):
        c = np.zeros(j + 1)
        c[j] = 1
        assert np.abs(Pi @ np.polynomial.legendre.legval(x, c)).max() < 1e-14


@pytest.mark.parametrize("N", [4, 5])
def test_projections(N):
    x, _ = basis.lgl_nodes_weights(N)
    P = basis.dg_to_fd_matrix(N, x)
    R = basis.fd_to_dg_matrix(N, x)
    xc = basis.subcell_centres(N)
    np.testing.assert_allclose(np.diff(xc), 2.0 / (2 * N + 1), atol=1e-15)
    for k in range(N + 1):
        np.testing.assert_allclose(P @ x ** k, xc ** k, atol=1e-13)   # exact evaluation
    for k in range(6):
        np.testing.assert_allclose(R @ xc ** k, x ** k, atol=1e-13)   # sixth-order interpolation
    np.testing.assert_allclose(R @ P, np.eye(N + 1), atol=1e-14)      # round trip
    # every row lives on 6 consecutive subcells around the node
    for j in range(N + 1):
        nz = np.nonzero(R[j])[0]
        assert nz.max() - nz.min() < 6
        nearest = np.argmin(np.abs(xc - x[j]))
        assert nz.min() <= nearest <= nz.max()


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7])
def test_filter_low_rank_form(N):
    """The DG kernels apply the filter as I - sum_m (1 - sigma_m) v_m w_m^T over
    the modes damped by more than 1e-20 (v_m the nodal values of mode m, w_m
    row m of V^-1).  That drops (1 - sigma_m) v_m w_m^T for the other modes, a
    change below 1e-20 per unit coefficient: the forms agree to rounding, and
    at the default a = 36, b = 50 only modes N-1 and N (N = 2: mode N; N = 6, 7:
    modes N-2 .. N) are kept."""
    x, _ = basis.lgl_nodes_weights(N)
    V = basis.vandermonde(N, x)
    Vi = np.linalg.inv(V)
    sig = basis.filter_sigma(N)
    damp = -np.expm1(-36.0 * (np.arange(N + 1) / N) ** 100)
    kept = [m for m in range(N + 1) if damp[m] > 1e-20]
    assert kept == list(range(N - {2: 0, 6: 2, 7: 2}.get(N, 1), N + 1))
    low = np.eye(N + 1) - sum(damp[m] * np.outer(V[:, m], Vi[m]) for m in kept)
    np.testing.assert_allclose(low, basis.filter_matrix(N, x), rtol=0, atol=1e-14)
    assert np.all(np.abs(1.0 - sig[[m for m in range(N + 1) if m not in kept]]) <= 1e-20)
