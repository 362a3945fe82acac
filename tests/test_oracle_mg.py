"""Pins of oracle/mg.py against facts fixed by the mathematics: nested DG spaces,
the Chebyshev error polynomial, symmetry of the V-cycle, convergence to the
exact discrete solution, and the minimal-residual property of GMRES."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.basis import gauss_lobatto_nodes
from oracle.mg import prolongation, jacobi_diagonal, chebyshev, VCycle, fgmres
from oracle.sipg import Mesh, assemble, BlockOperator, global_1d, lex_to_cell_major
from oracle.solve import FastDiag


def _nodal_values(k, nc, f):
    """Values of f at the Gauss-Lobatto nodes of every cell, cell-major layout."""
    n = k + 1
    x = gauss_lobatto_nodes(k)
    g = np.concatenate([(c + x) / nc for c in range(nc)]).reshape(nc, n)
    Z, Y, X = np.meshgrid(g.reshape(-1), g.reshape(-1), g.reshape(-1), indexing="ij")
    lex = f(X, Y, Z).reshape(-1)
    return lex[lex_to_cell_major(k, nc, nc, nc)]


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_prolongation_reproduces_coarse_polynomials(k):
    # a global polynomial of degree <= k per direction lies in both DG spaces
    rng = np.random.default_rng(k)
    c = rng.standard_normal((k + 1, k + 1, k + 1))
    f = lambda X, Y, Z: sum(c[a, b, d] * X ** a * Y ** b * Z ** d
                            for a in range(k + 1) for b in range(k + 1) for d in range(k + 1))
    P = prolongation(k, 2, 2, 2)
    coarse = _nodal_values(k, 2, f)
    fine = _nodal_values(k, 4, f)
    np.testing.assert_allclose(P @ coarse, fine, atol=1e-12 * np.abs(fine).max())


@pytest.mark.parametrize("k", [1, 2, 3])
def test_prolongation_preserves_the_l2_inner_product(k):
    # nested spaces: P^T M_fine P = M_coarse for the 3D DG mass matrix M (x) M (x) M
    def mass3(nc):
        M, _ = global_1d(k, nc)
        p = lex_to_cell_major(k, nc, nc, nc)
        return np.kron(M, np.kron(M, M))[np.ix_(p, p)]
    P = prolongation(k, 2, 2, 2).toarray()
    np.testing.assert_allclose(P.T @ mass3(4) @ P, mass3(2), atol=1e-13)


def test_jacobi_diagonal_is_the_matrix_diagonal():
    m = Mesh(3, 3, 3)
    for k in (1, 3):
        A = assemble(Mesh(3, 3, 3), k)
        np.testing.assert_allclose(jacobi_diagonal(k, 3, 3, 3), A.diagonal(), rtol=1e-14)


@pytest.mark.parametrize("degree", [1, 2, 3, 5])
def test_chebyshev_error_polynomial(degree):
    # with b = 0 the smoother maps an eigenvector v of D^{-1}A (A v = lam D v)
    # to p(lam) v, p(t) = T_m((theta - t)/delta) / T_m(theta/delta)
    k, nc = 2, 2
    A = assemble(Mesh(nc, nc, nc), k).toarray()
    D = np.diag(A)
    lam, V = sla.eigh(A, np.diag(D))
    lmax, ratio = 1.05 * lam[-1], 15.0
    lmin = lmax / ratio
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    T = np.polynomial.chebyshev.Chebyshev.basis(degree)
    for idx in (0, len(lam) // 2, len(lam) - 1):
        v = V[:, idx]
        out = chebyshev(lambda u: A @ u, 1.0 / D, np.zeros_like(v), v, lmax, degree, ratio)
        p = T((theta - lam[idx]) / delta) / T(theta / delta)
        np.testing.assert_allclose(out, p * v, atol=1e-12 * np.abs(v).max())


def test_vcycle_is_symmetric_and_converges():
    k, nc = 2, 4
    mg = VCycle(k, nc, coarse_nc=1, lmax=[None] + [2.9] * 2)
    A = BlockOperator(Mesh(nc, nc, nc), k)
    n = mg.levels[-1].ndofs
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal((2, n))
    assert abs(u @ mg(v) - v @ mg(u)) < 1e-11 * abs(u @ mg(v))
    b = rng.standard_normal(n)
    xs = FastDiag(k, nc, nc, nc).solve(b)
    x = np.zeros(n)
    errs = []
    for _ in range(8):
        x = x + mg(b - A.apply(x))
        errs.append(np.linalg.norm(x - xs) / np.linalg.norm(xs))
    assert errs[-1] < 1e-3 and errs[-1] < errs[0] * 1e-2


def test_gmres_minimal_residual_property():
    # identity preconditioner: after j steps x minimises ||b - A x|| over span{b, Ab, ...}
    rng = np.random.default_rng(3)
    n = 40
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(np.linspace(1, 30, n)) @ Q.T + 0.1 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    for j in (1, 3, 6):
        x, its, _ = fgmres(lambda v: A @ v, lambda v: v, b, rtol=1e-300, restart=j, maxit=j)
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(j)], axis=1)
        c = np.linalg.lstsq(A @ K, b, rcond=None)[0]
        assert its == j
        np.testing.assert_allclose(np.linalg.norm(b - A @ x), np.linalg.norm(b - A @ K @ c), rtol=1e-8)


def test_fgmres_with_vcycle_reaches_discrete_solution():
    k, nc = 3, 4
    mg = VCycle(k, nc, coarse_nc=1, lmax=[None] + [2.9] * 2)
    A = BlockOperator(Mesh(nc, nc, nc), k)
    b = np.random.default_rng(1).standard_normal(A.mesh.ncells * 64)
    x, its, hist = fgmres(A.apply, mg, b, rtol=1e-10)
    xs = FastDiag(k, nc, nc, nc).solve(b)
    assert hist[-1] <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8
    assert its < 30


@pytest.mark.parametrize("k", [1, 2])
def test_vcycle_without_smoothing_is_the_two_grid_correction(k):
    """One V-cycle over two levels with the smoother switched off and the exact coarse solve is
    x1 = x0 + P A_c^{-1} P^T (b - A x0), with A and A_c the matrices assembled on the fine and the
    coarse mesh (rediscretized, Algorithm 2) and the error e1 = (I - P A_c^{-1} P^T A) e0. Checked
    against dense linear algebra on the assembled matrices: a restriction by P instead of P^T, a
    scaled correction or a coarse operator of the wrong mesh would each fail."""
    nc = 4
    mg = VCycle(k, nc, coarse_nc=2)
    mg.smooth = lambda l, b, x, post=False: x  # no pre- or post-smoothing
    A = assemble(Mesh(nc, nc, nc), k).toarray()
    Ac = assemble(Mesh(2, 2, 2), k).toarray()
    P = prolongation(k, 2, 2, 2).toarray()
    rng = np.random.default_rng(7 + k)
    b, x0 = rng.standard_normal((2, A.shape[0]))
    x1 = mg.vcycle(1, b, x0)
    expect = x0 + P @ np.linalg.solve(Ac, P.T @ (b - A @ x0))
    np.testing.assert_allclose(x1, expect, rtol=0, atol=1e-11 * np.abs(expect).max())
    xs = np.linalg.solve(A, b)
    e0, e1 = xs - x0, xs - x1
    np.testing.assert_allclose(e1, e0 - P @ np.linalg.solve(Ac, P.T @ (A @ e0)), atol=1e-10 * np.abs(e0).max())
