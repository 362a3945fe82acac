"""Exact discrete Poisson solve, right-hand side and L2 error (Sec. 7.2).

Test infrastructure (see ``oracle/__init__``).

Sec. 7.2 solves Eq. (1) on the unit cube with the manufactured solution
u = sin(pi x) sin(pi y) sin(pi z), i.e. f = 3 pi^2 u and g = 0.

* ``fast_diag_solve``: the discrete solution u_h = A^{-1} b. With the 1D
  generalized eigenpairs L V = M V Lambda (V^T M V = I) of the global 1D
  factors of Eq. (9), A^{-1} = (V(x)V(x)V) diag(1/(l_i + l_j + l_m)) (V(x)V(x)V)^T.
  Pinned against scipy's sparse direct solver on the assembled matrix.
* ``rhs_sine``: b_a = int f phi_a; f is separable, so b = 3 pi^2 b1 (x) b1 (x) b1
  with b1 the 1D load vector of sin(pi x), integrated by 30-point Gauss per
  cell (exact to rounding for k <= 7).
* ``rhs_modes``: the same for a sum of sine modes (the batched problems);
  pinned against ``rhs_sine`` for the single mode (1, 1, 1) and against the
  closed-form integrals of the k = 1 basis for modes with p, q, r distinct
  (tests/test_oracle_basis.py).
* ``l2_error``: || u_h - u ||_L2 by per-cell tensor Gauss quadrature with k+4
  points per direction (the expanded form ||u_h||^2 - 2(u_h,u) + ||u||^2
  cancels to about 1e-8 and is not used). Pinned by the O(h^(k+1))
  convergence rate of the discrete solution.
"""
import numpy as np
import scipy.linalg as sla

from .basis import gauss_lobatto_nodes, gauss_legendre, lagrange_values
from .sipg import global_1d, lex_to_cell_major


def load_vector_1d(k, nc, func, length=1.0, q=30):
    """b1[c*n + i] = int_{cell c} func(x) phi_i(x) dx."""
    n = k + 1
    h = length / nc
    nodes = gauss_lobatto_nodes(k)
    xq, wq = gauss_legendre(q)
    phi = lagrange_values(nodes, xq)  # (q, n)
    b = np.zeros(nc * n)
    for c in range(nc):
        xs = (c + xq) * h
        b[c * n:(c + 1) * n] = h * (wq * func(xs)) @ phi
    return b


def rhs_sine(k, nx, ny, nz):
    """Load vector of f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), cell-major layout."""
    f1 = lambda s: np.sin(np.pi * s)
    bx = load_vector_1d(k, nx, f1)
    by = load_vector_1d(k, ny, f1)
    bz = load_vector_1d(k, nz, f1)
    lex = 3.0 * np.pi ** 2 * np.kron(bz, np.kron(by, bx))
    return lex[lex_to_cell_major(k, nx, ny, nz)]


def rhs_modes(k, nx, ny, nz, modes):
    """Load vector of f = sum_m a_m pi^2 (p^2+q^2+r^2) sin(p pi x) sin(q pi y) sin(r pi z).

    ``modes`` is a list of (a, p, q, r); the exact solution is
    sum_m a_m sin(p pi x) sin(q pi y) sin(r pi z).
    """
    lex = 0.0
    for a, p, q, r in modes:
        bx = load_vector_1d(k, nx, lambda s: np.sin(p * np.pi * s))
        by = load_vector_1d(k, ny, lambda s: np.sin(q * np.pi * s))
        bz = load_vector_1d(k, nz, lambda s: np.sin(r * np.pi * s))
        lex = lex + a * np.pi ** 2 * (p * p + q * q + r * r) * np.kron(bz, np.kron(by, bx))
    return lex[lex_to_cell_major(k, nx, ny, nz)]


class FastDiag:
    """Exact inverse of the Eq. (9) operator on a uniform box mesh."""

    def __init__(self, k, nx, ny, nz, pen="config", length=(1.0, 1.0, 1.0)):
        self.k, self.nc = k, (nx, ny, nz)
        self.eig = []
        for d, nc in enumerate((nx, ny, nz)):
            M, L = global_1d(k, nc, length[d], pen)
            lam, V = sla.eigh(L, M)
            self.eig.append((lam, V))
        self.perm = lex_to_cell_major(k, nx, ny, nz)

    def solve(self, b_cell):
        n = self.k + 1
        nx, ny, nz = self.nc
        lex = np.empty_like(b_cell)
        lex[self.perm] = b_cell
        T = lex.reshape(nz * n, ny * n, nx * n)
        (lx, Vx), (ly, Vy), (lz, Vz) = self.eig
        # T <- (Vz^T, Vy^T, Vx^T) T
        T = np.einsum("zyx,xa->zya", T, Vx, optimize=True)
        T = np.einsum("zya,yb->zba", T, Vy, optimize=True)
        T = np.einsum("zba,zc->cba", T, Vz, optimize=True)
        T = T / (lz[:, None, None] + ly[None, :, None] + lx[None, None, :])
        T = np.einsum("cba,xa->cbx", T, Vx, optimize=True)
        T = np.einsum("cbx,yb->cyx", T, Vy, optimize=True)
        T = np.einsum("cyx,zc->zyx", T, Vz, optimize=True)
        return T.reshape(-1)[self.perm]


def l2_error(u_cell, k, nx, ny, nz, exact, q=None):
    """|| u_h - exact ||_L2 on the unit cube, per-cell tensor Gauss, q = k+4."""
    n = k + 1
    q = q or k + 4
    nodes = gauss_lobatto_nodes(k)
    xq, wq = gauss_legendre(q)
    E = lagrange_values(nodes, xq)  # (q, n)
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    U = u_cell.reshape(nz, ny, nx, n, n, n)  # (cz, cy, cx, l, j, i)
    total = 0.0
    for cz in range(nz):
        Uz = U[cz]
        # values at quadrature points: (cy, cx, qz, qy, qx)
        V = np.einsum("yxlji,ai->yxlja", Uz, E, optimize=True)
        V = np.einsum("yxlja,bj->yxlba", V, E, optimize=True)
        V = np.einsum("yxlba,cl->yxcba", V, E, optimize=True)
        xs = (np.arange(nx)[:, None] + xq[None, :]) * h[0]   # (cx, qx)
        ys = (np.arange(ny)[:, None] + xq[None, :]) * h[1]
        zs = (cz + xq) * h[2]
        X = xs[None, :, None, None, :]
        Y = ys[:, None, None, :, None]
        Z = zs[None, None, :, None, None]
        ex = exact(X, Y, Z)
        W = (wq[:, None, None] * wq[None, :, None] * wq[None, None, :])[None, None]
        total += np.sum(W * (V - ex) ** 2) * h[0] * h[1] * h[2]
    return np.sqrt(total)


def sine_exact(x, y, z):
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
