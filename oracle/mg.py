"""Geometric multigrid V-cycle (Algorithm 2) with a Chebyshev-Jacobi smoother,
and flexible GMRES (Sec. 7), in FP64 on the CPU.

Test infrastructure (see ``oracle/__init__``).

What this restates
------------------
* Algorithm 2 (Sec. 7.1): at level l > 0 pre-smooth, form the residual,
  restrict it, recurse with a zero initial guess, prolongate and add the
  correction, post-smooth; at level 0 solve exactly.
* Levels: uniform refinement by 2 in every direction, the same degree k on
  every level, the operator rediscretized on each level (its h and penalty).
* Prolongation: the coarse DG space is nested in the fine one, so the fine
  coefficients of a coarse function are its values at the fine cells'
  Gauss-Lobatto nodes: per direction P1_c[i, j] = phi_j((c + x_i) / 2) for
  child c in {0, 1}, and in 3D the Kronecker product of the three 1D
  factors. Restriction is its transpose.
* Smoother, one of two: Chebyshev-Jacobi, ``degree`` steps of the Chebyshev
  semi-iteration for D^{-1} A on the interval [lmax / ratio, lmax], D = diag(A)
  (Saad, "Iterative Methods for Sparse Linear Systems", Alg. 12.1 with a Jacobi
  preconditioner; the eigenvalue bound lmax is an input); or the paper's
  vertex-patch multiplicative Schwarz smoother (oracle/schwarz.py), one sweep
  over the eight patch colours, ascending before and descending after the
  coarse-grid correction.
* Coarse solve: exact (fast diagonalization, oracle/solve.py).
* FGMRES (Saad 1993, right preconditioning, restart m): modified
  Gram-Schmidt Arnoldi, Givens rotations, stop when the Arnoldi residual
  norm |g_{j+1}| <= rtol * ||b - A x0||.

Pins (tests/test_oracle_mg.py): prolongation reproduces coarse polynomials
exactly; R = P^T; the smoother's error polynomial equals the scaled
Chebyshev polynomial on eigenvectors of D^{-1}A; one V-cycle with the exact
coarse solve and no smoothing reduces to the two-grid coarse correction
identity; FGMRES with the identity preconditioner equals GMRES (Krylov
minimal residual, checked against the normal equations on tiny systems).
"""
import numpy as np
import scipy.sparse as sp

from .basis import gauss_lobatto_nodes, lagrange_values
from .sipg import Mesh, BlockOperator, global_1d, lex_to_cell_major
from .solve import FastDiag
from .schwarz import VertexPatchSmoother


def prolongation_1d(k):
    """P1[c] (n x n): fine-child c coefficients from coarse coefficients."""
    x = gauss_lobatto_nodes(k)
    return [lagrange_values(x, (c + x) / 2.0) for c in (0, 1)]


def prolongation(k, ncx, ncy, ncz):
    """Sparse P: coarse mesh (ncx, ncy, ncz) -> fine mesh (2ncx, 2ncy, 2ncz), cell-major layouts."""
    n = k + 1
    nb = n ** 3
    P1 = prolongation_1d(k)
    rows, cols, vals = [], [], []
    fx, fy = 2 * ncx, 2 * ncy
    for cz in range(ncz):
        for cy in range(ncy):
            for cx in range(ncx):
                C = (cz * ncy + cy) * ncx + cx
                for bz in (0, 1):
                    for by in (0, 1):
                        for bx in (0, 1):
                            F = ((2 * cz + bz) * fy + (2 * cy + by)) * fx + (2 * cx + bx)
                            blk = np.kron(P1[bz], np.kron(P1[by], P1[bx]))
                            r, c = np.nonzero(np.abs(blk) > 0)
                            rows.append(F * nb + r)
                            cols.append(C * nb + c)
                            vals.append(blk[r, c])
    nf = 8 * ncx * ncy * ncz * nb
    nc = ncx * ncy * ncz * nb
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nf, nc))


def jacobi_diagonal(k, nx, ny, nz, pen="config"):
    """diag(A) from the Kronecker form of Eq. (9): diag(Lz)(x)diag(My)(x)diag(Mx) + ..."""
    dx = [np.diag(m) for m in global_1d(k, nx, pen=pen)]
    dy = [np.diag(m) for m in global_1d(k, ny, pen=pen)]
    dz = [np.diag(m) for m in global_1d(k, nz, pen=pen)]
    (mx, lx), (my, ly), (mz, lz) = dx, dy, dz
    lex = np.kron(lz, np.kron(my, mx)) + np.kron(mz, np.kron(ly, mx)) + np.kron(mz, np.kron(my, lx))
    return lex[lex_to_cell_major(k, nx, ny, nz)]


def chebyshev(apply_A, dinv, b, x, lmax, degree=3, ratio=15.0):
    """`degree` steps of Chebyshev-Jacobi on A x = b from x (returns the new x).

    Interval [lmax/ratio, lmax] for the spectrum of D^{-1} A.
    """
    lmin = lmax / ratio
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b - apply_A(x)
    d = dinv * r / theta
    x = x + d
    for _ in range(1, degree):
        r = r - apply_A(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        x = x + d
        rho = rho_new
    return x


class Level:
    def __init__(self, k, nc, pen="config"):
        self.k, self.nc = k, nc
        self.mesh = Mesh(nc, nc, nc)
        self.A = BlockOperator(self.mesh, k, pen)
        self.dinv = 1.0 / jacobi_diagonal(k, nc, nc, nc, pen)
        self.ndofs = self.mesh.ncells * (k + 1) ** 3


class VCycle:
    """Algorithm 2 on the cube, finest nc^3 cells, coarsest `coarse_nc`^3 cells."""

    def __init__(self, k, nc, coarse_nc=1, pen="config", degree=3, ratio=15.0, lmax=None, smoother="chebyshev"):
        self.k = k
        self.smoother = smoother
        sizes = [nc]
        while sizes[-1] > coarse_nc:
            if sizes[-1] % 2:
                raise ValueError("cells per direction must halve down to coarse_nc")
            sizes.append(sizes[-1] // 2)
        sizes = sizes[::-1]  # level 0 = coarsest
        self.levels = [Level(k, s, pen) for s in sizes]
        self.P = [None] + [prolongation(k, s, s, s) for s in sizes[:-1]]
        self.coarse = FastDiag(k, sizes[0], sizes[0], sizes[0], pen)
        self.degree, self.ratio = degree, ratio
        self.lmax = lmax if lmax is not None else [None] * len(sizes)
        self.vp = None
        if smoother == "vertex_patch":
            from .sipg import assemble
            self.vp = [None] + [VertexPatchSmoother(assemble(Mesh(s, s, s), k, pen), k, (s, s, s))
                                for s in sizes[1:]]
        elif smoother != "chebyshev":
            raise ValueError("smoother is 'chebyshev' or 'vertex_patch'")

    def smooth(self, l, b, x, post=False):
        if self.vp is not None:
            return self.vp[l].smooth(x, b, reverse=post)
        lev = self.levels[l]
        return chebyshev(lev.A.apply, lev.dinv, b, x, self.lmax[l], self.degree, self.ratio)

    def vcycle(self, l, b, x):
        if l == 0:
            return self.coarse.solve(b)
        lev = self.levels[l]
        x = self.smooth(l, b, x)
        r = b - lev.A.apply(x)
        rc = self.P[l].T @ r
        xc = self.vcycle(l - 1, rc, np.zeros_like(rc))
        x = x + self.P[l] @ xc
        return self.smooth(l, b, x, post=True)

    def __call__(self, b):
        return self.vcycle(len(self.levels) - 1, b, np.zeros_like(b))


def fgmres(apply_A, precond, b, rtol=1e-10, restart=30, maxit=200, x0=None):
    """Flexible GMRES with right preconditioning (Saad 1993), MGS Arnoldi.

    Returns (x, iterations, residual history relative to ||b - A x0||).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x)
    beta0 = np.linalg.norm(r)
    hist = [1.0]
    its = 0
    if beta0 == 0.0:
        return x, 0, hist
    while its < maxit:
        beta = np.linalg.norm(r)
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j_end = 0
        for j in range(restart):
            z = precond(V[j])
            Z.append(z)
            w = apply_A(z)
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / beta0)
            if abs(g[j + 1]) <= rtol * beta0 or its >= maxit:
                break
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_end] @ y[i + 1:j_end]) / H[i, i]
        for i in range(j_end):
            x = x + y[i] * Z[i]
        r = b - apply_A(x)
        if np.linalg.norm(r) <= rtol * beta0 * 1.0001 or abs(g[j_end]) <= rtol * beta0:
            break
    return x, its, hist
