"""Pins of the oracle's 1D basis (Sec. II-B) against closed forms and library routines.

Each test fixes the oracle to something other than itself: textbook closed forms of the
GLL nodes and weights, numpy's independent Legendre implementation, exact polynomial
calculus, and the textbook closed form of the GLL differentiation matrix.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg


@pytest.mark.parametrize("N,nodes,weights", [
    (1, [-1, 1], [1, 1]),
    (2, [-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    (3, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    (4, [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
    (5, [-1, -np.sqrt(1 / 3 + 2 * np.sqrt(7) / 21), -np.sqrt(1 / 3 - 2 * np.sqrt(7) / 21),
         np.sqrt(1 / 3 - 2 * np.sqrt(7) / 21), np.sqrt(1 / 3 + 2 * np.sqrt(7) / 21), 1],
     [1 / 15, (14 - np.sqrt(7)) / 30, (14 + np.sqrt(7)) / 30, (14 + np.sqrt(7)) / 30,
      (14 - np.sqrt(7)) / 30, 1 / 15]),
])
def test_gll_closed_forms(oracle, N, nodes, weights):
    """Closed-form Lobatto nodes and weights for N = 1..5 (Abramowitz & Stegun 25.4.32)."""
    x, w = oracle.gll_points_weights(N)
    np.testing.assert_allclose(x, nodes, atol=1e-15)
    np.testing.assert_allclose(w, weights, rtol=1e-14)


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_nodes_are_lobatto_roots(oracle, N):
    """Interior nodes are the roots of P_N' (numpy's own Legendre series), endpoints +-1."""
    x, _ = oracle.gll_points_weights(N)
    ref = np.sort(npleg.Legendre.basis(N).deriv().roots().real) if N > 1 else np.array([])
    np.testing.assert_allclose(x[1:-1], ref, atol=1e-13)
    assert x[0] == -1.0 and x[-1] == 1.0


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_quadrature_exactness(oracle, N):
    """GLL quadrature integrates x^k exactly for k <= 2N-1 and not for k = 2N."""
    x, w = oracle.gll_points_weights(N)
    for k in range(2 * N):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-13
    k = 2 * N
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-10
    assert abs(w.sum() - 2.0) < 1e-13


@pytest.mark.parametrize("n", range(2, 12))
def test_lagrange_kronecker(oracle, n):
    """l_i(xi_j) = delta_ij (Sec. II-B, Kronecker property)."""
    xi, _ = oracle.gll_points_weights(n - 1)
    np.testing.assert_allclose(oracle.lagrange_basis(xi, xi), np.eye(n), atol=1e-13)


@pytest.mark.parametrize("n", range(2, 12))
def test_hprime_exact_on_polynomials(oracle, n):
    """hprime differentiates every polynomial of degree <= N exactly at the nodes, and
    does not for degree N+1; rows sum to zero (derivative of a constant)."""
    N = n - 1
    xi, _ = oracle.gll_points_weights(N)
    H = oracle.lagrange_derivative_matrix(xi)
    for m in range(N + 1):
        np.testing.assert_allclose(H @ xi ** m, m * xi ** max(m - 1, 0) * (m > 0), atol=1e-11)
    err = H @ xi ** (N + 1) - (N + 1) * xi ** N
    assert np.max(np.abs(err)) > 1e-6
    np.testing.assert_allclose(H.sum(axis=1), 0.0, atol=1e-11)


@pytest.mark.parametrize("n", range(2, 12))
def test_hprime_textbook_closed_form(oracle, n):
    """GLL differentiation matrix closed form (Canuto et al., Spectral Methods, 2.3.28):
    D_il = P_N(xi_i) / (P_N(xi_l) (xi_i - xi_l)) for i != l, D_00 = -N(N+1)/4,
    D_NN = N(N+1)/4, other diagonal entries 0. P_N from numpy's Legendre series."""
    N = n - 1
    xi, _ = oracle.gll_points_weights(N)
    P = npleg.legval(xi, [0] * N + [1])
    D = np.zeros((n, n))
    for i in range(n):
        for l in range(n):
            if i != l:
                D[i, l] = P[i] / (P[l] * (xi[i] - xi[l]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    np.testing.assert_allclose(oracle.lagrange_derivative_matrix(xi), D, atol=1e-11)


def test_min_spacing_shrinks_like_n_minus_2(oracle):
    """Sec. IV-B: the smallest GLL spacing decreases as O(N^-2). Asymptotically
    1 - xi_{N-1} -> j_{1,1}^2 / (2 N^2), j_{1,1} the first zero of the Bessel function J_1
    (Bessel-zero asymptotics of Legendre zeros; scipy supplies j_{1,1})."""
    from scipy.special import jn_zeros
    limit = jn_zeros(1, 1)[0] ** 2 / 2.0
    ratios = []
    for N in (4, 8, 16, 32, 64):
        xi, _ = oracle.gll_points_weights(N)
        ratios.append(np.min(np.diff(xi)) * N * N)
    assert all(a < b for a, b in zip(ratios, ratios[1:]))
    assert all(5.0 < r < limit for r in ratios)
    assert abs(ratios[-1] / limit - 1.0) < 0.02


def test_ricker_closed_form(oracle):
    """Ricker wavelet: R(t0) = 1, zeros at t0 +- 1/(pi f0 sqrt 2), minima -2 exp(-3/2) at
    t0 +- sqrt(3/2)/(pi f0), and zero integral over a long window."""
    f0, t0 = 10.0, 0.12
    assert oracle.ricker(t0, f0, t0) == 1.0
    z = 1.0 / (np.pi * f0 * np.sqrt(2.0))
    np.testing.assert_allclose(oracle.ricker([t0 - z, t0 + z], f0, t0), 0.0, atol=1e-15)
    tm = np.sqrt(1.5) / (np.pi * f0)
    np.testing.assert_allclose(oracle.ricker(t0 + tm, f0, t0), -2 * np.exp(-1.5), rtol=1e-14)
    t = np.linspace(-1.0, 1.24, 200001)
    assert abs(np.trapezoid(oracle.ricker(t, f0, t0), t)) < 1e-10


def test_dispersion_error_definition(oracle):
    """Sec. V-C-1 error is the ratio of squared L2 norms: 0 for the exact waveform, 1 for
    a zero waveform, s^2 for a waveform scaled by (1 + s)."""
    t = np.linspace(0, 1, 1001)
    wt = np.sin(7 * t) * np.exp(-t)
    assert oracle.dispersion_error(wt, wt) == 0.0
    assert abs(oracle.dispersion_error(0 * wt, wt) - 1.0) < 1e-15
    assert abs(oracle.dispersion_error(1.1 * wt, wt) - 0.01) < 1e-12
