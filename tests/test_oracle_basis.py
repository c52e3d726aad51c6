"""Pins of the oracle's 1D GLL building blocks against closed forms (no GPU)."""

import math

import numpy as np
import pytest

from oracle import gll


@pytest.mark.parametrize(
    "r,nodes,weights",
    [
        (1, [-1, 1], [1, 1]),
        (2, [-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
        (3, [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
        (4, [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
    ],
)
def test_gll_closed_forms(r, nodes, weights):
    x, w = gll.gll(r)
    assert np.allclose(x, nodes, atol=1e-15, rtol=0)
    assert np.allclose(w, weights, atol=1e-15, rtol=0)


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6])
def test_gll_exactness(r):
    """GLL with r+1 points integrates x^k exactly for k <= 2r-1, not for k = 2r."""
    x, w = gll.gll(r)
    assert np.allclose(x, -x[::-1], atol=1e-15)
    for k in range(2 * r):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    k = 2 * r
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_derivative_exact_on_polynomials(r):
    x, _ = gll.gll(r)
    D = gll.derivative_matrix(r)
    for k in range(r + 1):
        assert np.allclose(D @ x ** k, k * x ** max(k - 1, 0) if k else 0 * x, atol=1e-13)
    assert np.allclose(D.sum(axis=1), 0, atol=1e-13)


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_summation_by_parts(r):
    """W D + D^T W = diag(-1, 0, ..., 0, 1) for collocated GLL."""
    x, w = gll.gll(r)
    D = gll.derivative_matrix(r)
    W = np.diag(w)
    B = np.zeros((r + 1, r + 1))
    B[0, 0], B[-1, -1] = -1, 1
    assert np.allclose(W @ D + D.T @ W, B, atol=1e-13)


@pytest.mark.parametrize("r", [2, 3, 5])
def test_lagrange_interpolation_and_subintervals(r):
    """Interpolation is exact for degree <= r, including onto each 2:1 half interval."""
    x, _ = gll.gll(r)
    rng = np.random.default_rng(r)
    coef = rng.standard_normal(r + 1)
    f = lambda t: np.polyval(coef, t)
    pts = rng.uniform(-1, 1, 17)
    assert np.allclose(gll.lagrange_eval(x, pts) @ f(x), f(pts), atol=1e-13)
    for s in (0, 1):
        half = 0.5 * (x + (2 * s - 1))
        assert np.allclose(gll.lagrange_eval(x, half) @ f(x), f(half), atol=1e-13)
    Ld = gll.lagrange_deriv_eval(x, pts)
    assert np.allclose(Ld @ f(x), np.polyval(np.polyder(coef), pts), atol=1e-12)
