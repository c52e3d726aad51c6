"""1D Gauss-Lobatto-Legendre nodes, weights and Lagrange operators (test oracle).

The paper's DG discretisation (Sec. 2) is read as a nodal Lagrange basis on
the n = r+1 Gauss-Lobatto-Legendre points per direction with collocated
quadrature; these are the 1D building blocks, written from their textbook
definitions.
"""

import numpy as np


def legendre(r, x):
    """P_r(x) by Bonnet's recurrence (k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2})."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if r == 0:
        return p_prev
    p = x.copy()
    for k in range(2, r + 1):
        p_prev, p = p, ((2 * k - 1) * x * p - (k - 1) * p_prev) / k
    return p


def legendre_dp(r, x):
    """P_r'(x) = r (P_{r-1} - x P_r) / (1 - x^2), valid for |x| < 1."""
    x = np.asarray(x, dtype=np.float64)
    return r * (legendre(r - 1, x) - x * legendre(r, x)) / (1.0 - x * x)


def gll(r):
    """Nodes (ascending) and weights of the (r+1)-point GLL rule on [-1, 1].

    Interior nodes are the roots of P_r', found by Newton's method from the
    Chebyshev-Gauss-Lobatto points; weights are 2 / (r (r+1) P_r(x)^2).
    """
    if r < 1:
        raise ValueError("degree must be >= 1")
    x = -np.cos(np.pi * np.arange(r + 1) / r)
    x[0], x[-1] = -1.0, 1.0
    interior = x[1:-1].copy()
    for _ in range(100):
        dp = legendre_dp(r, interior)
        # Legendre ODE: (1 - x^2) P'' = 2 x P' - r (r+1) P
        d2p = (2 * interior * dp - r * (r + 1) * legendre(r, interior)) / (1 - interior ** 2)
        step = dp / d2p
        interior = interior - step
        if np.all(np.abs(step) < 1e-16):
            break
    x[1:-1] = interior
    w = 2.0 / (r * (r + 1) * legendre(r, x) ** 2)
    return x, w


def lagrange_eval(nodes, pts):
    """L[k, j] = l_j(pts[k]) for the Lagrange basis on ``nodes`` (product formula)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.atleast_1d(np.asarray(pts, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(pts), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (pts - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_deriv_eval(nodes, pts):
    """Ld[k, j] = l_j'(pts[k]): sum over the dropped factor of the product rule."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.atleast_1d(np.asarray(pts, dtype=np.float64))
    n = len(nodes)
    Ld = np.zeros((len(pts), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(pts), 1.0 / (nodes[j] - nodes[m]))
            for l in range(n):
                if l != j and l != m:
                    term *= (pts - nodes[l]) / (nodes[j] - nodes[l])
            Ld[:, j] += term
    return Ld


def derivative_matrix(r):
    """D[k, j] = l_j'(x_k) at the GLL nodes of degree r."""
    x, _ = gll(r)
    return lagrange_deriv_eval(x, x)
