"""Pins of oracle/basis.py: properties fixed by the mathematics, not by the oracle."""
import numpy as np
import pytest

from oracle.basis import (gauss_lobatto_nodes, gauss_legendre, lagrange_values,
                          lagrange_derivatives, differentiation_matrix)
from oracle.sipg import Ref1D


def test_gauss_lobatto_closed_forms():
    # Gauss-Lobatto points on [-1, 1]: k=2: 0; k=3: +-1/sqrt(5); k=4: 0, +-sqrt(3/7)
    to01 = lambda t: (np.asarray(t) + 1.0) / 2.0
    np.testing.assert_allclose(gauss_lobatto_nodes(1), [0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(gauss_lobatto_nodes(2), [0.0, 0.5, 1.0], atol=1e-15)
    s5 = 1 / np.sqrt(5)
    np.testing.assert_allclose(gauss_lobatto_nodes(3), to01([-1, -s5, s5, 1]), atol=1e-15)
    s = np.sqrt(3 / 7)
    np.testing.assert_allclose(gauss_lobatto_nodes(4), to01([-1, -s, 0, s, 1]), atol=1e-15)


@pytest.mark.parametrize("k", range(1, 16))
def test_gauss_lobatto_exactness(k):
    # The (k+1)-point Lobatto rule with these nodes integrates degree 2k-1 exactly;
    # its weights are int phi_i, so integrating monomials checks the nodes.
    x = gauss_lobatto_nodes(k)
    xq, wq = gauss_legendre(k + 2)
    w = wq @ lagrange_values(x, xq)
    for p in range(2 * k):
        assert abs(w @ x ** p - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("q", range(1, 20))
def test_gauss_legendre_exactness(q):
    x, w = gauss_legendre(q)
    for p in range(2 * q):
        assert abs(w @ x ** p - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("k", range(1, 16))
def test_lagrange_reproduces_polynomials(k):
    nodes = gauss_lobatto_nodes(k)
    pts = np.random.default_rng(k).uniform(0, 1, 17)
    V = lagrange_values(nodes, pts)
    dV = lagrange_derivatives(nodes, pts)
    np.testing.assert_allclose(lagrange_values(nodes, nodes), np.eye(k + 1), atol=1e-15)
    for p in range(k + 1):
        np.testing.assert_allclose(V @ nodes ** p, pts ** p, atol=1e-13)
        dexact = p * pts ** (p - 1) if p > 0 else 0 * pts
        np.testing.assert_allclose(dV @ nodes ** p, dexact, atol=1e-11)
    np.testing.assert_allclose(differentiation_matrix(nodes).sum(axis=1), 0, atol=1e-11)


def test_k1_textbook_matrices():
    r = Ref1D(1)
    np.testing.assert_allclose(r.Mhat, [[1 / 3, 1 / 6], [1 / 6, 1 / 3]], atol=1e-15)
    np.testing.assert_allclose(r.Khat, [[1, -1], [-1, 1]], atol=1e-14)
    np.testing.assert_allclose(r.d0, [-1, 1], atol=1e-14)
    np.testing.assert_allclose(r.d1, [-1, 1], atol=1e-14)


@pytest.mark.parametrize("k", range(1, 16))
def test_reference_matrices_integrals(k):
    r = Ref1D(k)
    x = r.nodes
    # coefficients of x^p are its nodal values; 1^T Mhat c = int x^p, c^T Mhat c = int x^2p
    for p in range(k + 1):
        c = x ** p
        assert abs(np.ones(k + 1) @ r.Mhat @ c - 1 / (p + 1)) < 1e-13
        assert abs(c @ r.Mhat @ c - 1 / (2 * p + 1)) < 1e-13
        if p >= 1:
            assert abs(c @ r.Khat @ c - p * p / (2 * p - 1)) < 1e-11
    np.testing.assert_allclose(r.Khat @ np.ones(k + 1), 0, atol=1e-11)
    np.testing.assert_allclose(r.v0, np.eye(k + 1)[0], atol=1e-15)
    np.testing.assert_allclose(r.v1, np.eye(k + 1)[-1], atol=1e-15)
