"""Pins for the oracle's GLL nodes/weights and derivative matrix.

The paper (Sec. III.A) names n GLL points per direction, n = degree + 1, and
Listing 1 uses the derivative matrix dxm1 and its transpose dxtm1.  These
tests tie the oracle to closed forms, quadrature exactness and library
routines, none of which share code with it.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as L

NS = list(range(2, 17))


@pytest.mark.parametrize("n", NS)
def test_gll_nodes_are_lobatto_points(oracle, n):
    xi, w = oracle.gll(n)
    N = n - 1
    assert xi[0] == -1.0 and xi[-1] == 1.0
    assert np.all(np.diff(xi) > 0)
    # symmetric nodes
    np.testing.assert_allclose(xi, -xi[::-1], atol=2e-16)
    # interior nodes are the roots of P_N' (library routine)
    if N >= 2:
        roots = np.sort(L.Legendre.basis(N).deriv().roots().real)
        np.testing.assert_allclose(xi[1:-1], roots, atol=1e-12)
    # weights: 2 / (N (N+1) P_N(xi)^2) from the library's P_N
    PN = L.legval(xi, [0] * N + [1])
    np.testing.assert_allclose(w, 2.0 / (N * (N + 1) * PN ** 2), rtol=1e-12)


@pytest.mark.parametrize("n", NS)
def test_gll_quadrature_exactness(oracle, n):
    xi, w = oracle.gll(n)
    N = n - 1
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * N):          # exact for degree <= 2N - 1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, xi ** k) - exact) < 1e-13, k
    # and not exact at degree 2N (sanity: the rule really is Lobatto's)
    k = 2 * N
    assert abs(np.dot(w, xi ** k) - 2.0 / (k + 1)) > 1e-10


def test_gll_closed_forms(oracle):
    # Textbook Lobatto rules (Abramowitz & Stegun 25.4.32).
    xi, w = oracle.gll(3)
    np.testing.assert_allclose(xi, [-1, 0, 1], atol=1e-16)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-15)
    xi, w = oracle.gll(4)
    a = 1 / math.sqrt(5)
    np.testing.assert_allclose(xi, [-1, -a, a, 1], rtol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-15)
    xi, w = oracle.gll(5)
    b = math.sqrt(3 / 7)
    np.testing.assert_allclose(xi, [-1, -b, 0, b, 1], atol=1e-16)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-15)


def barycentric_dmat(x):
    """Lagrange derivative matrix from barycentric weights (Berrut &
    Trefethen 2004): D_ij = (lam_j / lam_i) / (x_i - x_j), D_ii = -sum."""
    n = len(x)
    lam = np.array([1.0 / np.prod([x[j] - x[k] for k in range(n) if k != j]) for j in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (x[i] - x[j])
        D[i, i] = -D[i].sum()
    return D


@pytest.mark.parametrize("n", NS)
def test_dmat_differentiates_polynomials(oracle, n):
    xi, _ = oracle.gll(n)
    D = oracle.dmat(xi)
    N = n - 1
    scale = np.abs(D).sum(axis=1).max()
    # D * 1 = 0
    assert np.abs(D @ np.ones(n)).max() < 1e-13 * scale
    # D * x^m = m x^(m-1) exactly for m <= N
    for m in range(1, N + 1):
        got = D @ xi ** m
        want = m * xi ** (m - 1)
        assert np.abs(got - want).max() < 2e-13 * scale * max(1, m), m
    # centro-antisymmetry of the GLL derivative matrix
    np.testing.assert_allclose(D, -D[::-1, ::-1], atol=1e-13 * scale)
    # corner entries -N(N+1)/4 and N(N+1)/4
    assert D[0, 0] == -N * (N + 1) / 4 and D[N, N] == N * (N + 1) / 4
    # independent barycentric formula
    np.testing.assert_allclose(D, barycentric_dmat(xi), atol=1e-12 * scale)
