"""1D Lagrange basis on Gauss-Lobatto points and Gauss-Legendre quadrature.

Test infrastructure (see ``oracle/__init__``).

Sec. 2: the shape functions are tensor products of 1D Lagrange interpolation
polynomials of degree k whose nodes are the k+1 Gauss-Lobatto points of the
reference interval [0, 1] (the reference cell is [0,1]^3).

Pinned by tests/test_oracle_basis.py: nodal property, partition of unity,
exact reproduction of monomials up to degree k, derivative check against
monomial derivatives, closed-form Gauss-Lobatto nodes for k = 2, 3, 4 and
the k = 1 textbook mass/stiffness matrices.
"""
import numpy as np
from numpy.polynomial import legendre as _leg


def gauss_lobatto_nodes(k):
    """k+1 Gauss-Lobatto points on [0, 1], ascending (Sec. 2).

    On [-1, 1] they are the end points and the roots of P_k', the derivative
    of the Legendre polynomial of degree k.
    """
    if k < 1:
        raise ValueError("degree k must be >= 1")
    interior = np.zeros(0)
    if k >= 2:
        coeffs = np.zeros(k + 1)
        coeffs[k] = 1.0
        interior = np.sort(np.real(_leg.legroots(_leg.legder(coeffs))))
    t = np.concatenate(([-1.0], interior, [1.0]))
    x = 0.5 * (t + 1.0)
    x[0], x[-1] = 0.0, 1.0
    return x


def gauss_legendre(q):
    """q-point Gauss-Legendre rule on [0, 1] (points ascending, weights sum to 1)."""
    t, w = _leg.leggauss(q)
    return 0.5 * (t + 1.0), 0.5 * w


def barycentric_weights(nodes):
    """w_j = 1 / prod_{m != j} (x_j - x_m)."""
    n = len(nodes)
    w = np.ones(n)
    for j in range(n):
        for m in range(n):
            if m != j:
                w[j] /= nodes[j] - nodes[m]
    return w


def lagrange_values(nodes, x):
    """phi_j(x) for all nodes j and all points x: array (len(x), n).

    Second (true) barycentric form; a point that coincides with a node gets
    the Kronecker delta exactly.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    w = barycentric_weights(nodes)
    out = np.zeros((len(x), len(nodes)))
    for p, xp in enumerate(x):
        diff = xp - nodes
        hit = np.nonzero(diff == 0.0)[0]
        if len(hit):
            out[p, hit[0]] = 1.0
            continue
        t = w / diff
        out[p] = t / t.sum()
    return out


def differentiation_matrix(nodes):
    """D[i, j] = phi_j'(x_i) (nodal differentiation matrix)."""
    n = len(nodes)
    w = barycentric_weights(nodes)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (nodes[i] - nodes[j])
        D[i, i] = -D[i].sum()
    return D


def lagrange_derivatives(nodes, x):
    """phi_j'(x) for all j at points x: array (len(x), n).

    phi_j' has degree k-1, so it equals its own interpolant on the nodes:
    phi_j'(x) = sum_i phi_j'(x_i) phi_i(x).
    """
    return lagrange_values(nodes, x) @ differentiation_matrix(nodes)
