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


def test_rhs_modes_single_mode_is_the_paper_right_hand_side():
    from oracle.solve import rhs_modes, rhs_sine
    for k, dims in ((1, (3, 4, 2)), (3, (2, 2, 3))):
        np.testing.assert_allclose(rhs_modes(k, *dims, [(1.0, 1, 1, 1)]), rhs_sine(k, *dims), rtol=1e-14, atol=0)


def test_rhs_modes_against_closed_form_integrals_k1():
    """k = 1: the Gauss-Lobatto basis on a cell [a, a + h] is phi_0 = (a + h - x)/h, phi_1 = (x - a)/h,
    whose integrals against sin(w x) have closed forms; the load vector of
    f = a pi^2 (p^2 + q^2 + r^2) sin(p pi x) sin(q pi y) sin(r pi z) is their tensor product, placed at
    g = ((cz ny + cy) nx + cx) 8 + (l 2 + j) 2 + i. Two modes with p, q, r all different."""
    from oracle.solve import rhs_modes

    def b1(w, nc):
        h = 1.0 / nc
        out = np.zeros((nc, 2))
        for c in range(nc):
            a = c * h
            s = (np.sin(w * (a + h)) - np.sin(w * a)) / (h * w * w)
            out[c, 0] = np.cos(w * a) / w - s
            out[c, 1] = -np.cos(w * (a + h)) / w + s
        return out

    nx, ny, nz = 3, 2, 4
    modes = [(0.7, 1, 2, 3), (-1.3, 3, 1, 2)]
    expect = np.zeros(nx * ny * nz * 8)
    for a, p, q, r in modes:
        bx, by, bz = b1(p * np.pi, nx), b1(q * np.pi, ny), b1(r * np.pi, nz)
        coef = a * np.pi ** 2 * (p * p + q * q + r * r)
        for cz in range(nz):
            for cy in range(ny):
                for cx in range(nx):
                    for l in range(2):
                        for j in range(2):
                            for i in range(2):
                                g = ((cz * ny + cy) * nx + cx) * 8 + (l * 2 + j) * 2 + i
                                expect[g] += coef * bx[cx, i] * by[cy, j] * bz[cz, l]
    got = rhs_modes(1, nx, ny, nz, modes)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-13 * np.abs(expect).max())
