"""Pins of oracle/sipg.py and oracle/solve.py against facts the paper and the
mathematics fix: brute-force quadrature of Eq. (2), a hand-worked k = 1
matrix, symmetry, definiteness, the spectral form of Eq. (9), the
O(h^(k+1)) convergence of the discrete solution and the paper's Table 3."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle.brute import assemble_dense
from oracle.sipg import (Mesh, assemble, BlockOperator, global_1d, kron_apply, lex_to_cell_major,
                         penalty, Ref1D)
from oracle.solve import FastDiag, rhs_sine, l2_error, sine_exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2)])
def test_kronecker_assembly_matches_brute_force(k, dims):
    m = Mesh(*dims)
    assert _rel(assemble(m, k).toarray(), assemble_dense(m, k)) < 1e-13


@pytest.mark.parametrize("pen", ["config", "paper"])
def test_brute_force_anisotropic_cells(pen):
    m = Mesh(2, 1, 1, lx=0.7, ly=1.3, lz=0.4)
    assert _rel(assemble(m, 2, pen).toarray(), assemble_dense(m, 2, pen)) < 1e-13


def test_brute_force_k7_one_cell():
    m = Mesh(1, 1, 1)
    assert _rel(assemble(m, 7).toarray(), assemble_dense(m, 7)) < 1e-13


def test_brute_force_k8_one_cell():
    # the first degree of the arbitrary-size range (n = 9): 3D quadrature of Eq. (2), 729 x 729
    m = Mesh(1, 1, 1)
    assert _rel(assemble(m, 8).toarray(), assemble_dense(m, 8)) < 1e-13


def test_hand_worked_k1_one_cell():
    rows = np.loadtxt(os.path.join(GOLDEN, "sipg_k1_one_cell_1d.txt"))
    for h in (1.0, 0.25):
        g = penalty(1, h)
        want = np.zeros((2, 2))
        for r, c, cg, ch in rows:
            want[int(r), int(c)] = cg * g + ch / h
        _, L = global_1d(1, 1, length=h)
        np.testing.assert_allclose(L, want, atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_symmetry_and_definiteness(k):
    m = Mesh(3, 2, 2)
    A = assemble(m, k)
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal((2, A.shape[0]))
    assert abs(u @ (A @ v) - v @ (A @ u)) < 1e-12 * abs(u @ (A @ v)) + 1e-12
    Ad = A.toarray()
    sla.cholesky(Ad)  # raises if not positive definite
    assert np.abs(A @ np.ones(A.shape[0])).max() > 1.0  # Dirichlet: constants are not in the kernel


@pytest.mark.parametrize("pen", ["config", "paper"])
@pytest.mark.parametrize("k", [1, 3, 7])
def test_1d_lowest_eigenvalue_tends_to_pi_squared(k, pen):
    # -u'' = lam u, u(0)=u(1)=0 has lowest eigenvalue pi^2
    M, L = global_1d(k, 16, pen=pen)
    lam = sla.eigh(L, M, eigvals_only=True)[0]
    assert abs(lam - np.pi ** 2) < max((1 / 16) ** (k + 1), 1e-11) * np.pi ** 2


@pytest.mark.parametrize("k", [2, 3])
def test_spectral_closed_form(k):
    nx, ny, nz = 3, 2, 4
    A = assemble(Mesh(nx, ny, nz), k)
    eig = []
    for nc in (nx, ny, nz):
        M, L = global_1d(k, nc)
        lam, V = sla.eigh(L, M)
        eig.append((M, lam, V))
    perm = lex_to_cell_major(k, nx, ny, nz)
    (Mx, lx, Vx), (My, ly, Vy), (Mz, lz, Vz) = eig
    for (a, b, c) in [(0, 0, 0), (1, 0, 2), (5, 3, 7)]:
        v = np.kron(Vz[:, c], np.kron(Vy[:, b], Vx[:, a]))[perm]
        w = (lx[a] + ly[b] + lz[c]) * np.kron(Mz @ Vz[:, c], np.kron(My @ Vy[:, b], Mx @ Vx[:, a]))[perm]
        assert _rel(A @ v, w) < 1e-12


@pytest.mark.parametrize("k,dims,lengths,pen", [
    (1, (3, 2, 4), (1.0, 1.0, 1.0), "config"), (2, (4, 3, 2), (0.7, 1.9, 0.45), "paper"),
    (3, (2, 3, 1), (1.0, 1.0, 1.0), "config"), (5, (1, 2, 3), (1.3, 0.6, 1.0), "config")])
def test_kron_apply_matches_assembled_matrix(k, dims, lengths, pen):
    # Kronecker-sum form of Eq. (9) (global 1D factors) against the element + face assembly
    A = assemble(Mesh(*dims, *lengths), k, pen)
    x = np.random.default_rng(k).uniform(-1, 1, A.shape[0])
    assert _rel(kron_apply(x, k, dims, lengths, pen), A @ x) < 1e-14


def test_kron_apply_matches_block_operator_k8():
    # element/face block rows (pinned to quadrature at k = 8 above) against the Kronecker sum
    dims = (2, 1, 3)
    bo = BlockOperator(Mesh(*dims), 8)
    x = np.random.default_rng(8).uniform(-1, 1, 6 * 9 ** 3)
    assert _rel(kron_apply(x, 8, dims), bo.apply(x)) < 1e-13


@pytest.mark.parametrize("k", [11, 15])
def test_high_degree_1d_lowest_eigenvalue(k):
    # the face terms of the global 1D stiffness at high degree: lowest eigenvalue of
    # -u'' = lam u with u(0) = u(1) = 0 on 3 cells is pi^2 to spectral accuracy
    M, L = global_1d(k, 3)
    lam = sla.eigh(L, M, eigvals_only=True)[0]
    assert abs(lam - np.pi ** 2) < 1e-9 * np.pi ** 2


@pytest.mark.parametrize("k", [12, 15])
def test_kron_apply_spectral_closed_form_high_degree(k):
    # tensor products of 1D generalized eigenvectors V (L V = M V diag(lam)) are mapped to
    # (lam_a + lam_b + lam_c) M v: checks the index order of the Kronecker sum on an anisotropic mesh
    dims = (3, 1, 2)
    eig = []
    for nc in dims:
        M, L = global_1d(k, nc)
        lam, V = sla.eigh(L, M)
        eig.append((M, lam, V))
    perm = lex_to_cell_major(k, *dims)
    (Mx, lx, Vx), (My, ly, Vy), (Mz, lz, Vz) = eig
    for (a, b, c) in [(0, 0, 0), (5, 3, 7), (30, 2, 19)]:
        v = np.kron(Vz[:, c], np.kron(Vy[:, b], Vx[:, a]))[perm]
        w = (lx[a] + ly[b] + lz[c]) * np.kron(Mz @ Vz[:, c], np.kron(My @ Vy[:, b], Mx @ Vx[:, a]))[perm]
        assert _rel(kron_apply(v, k, dims), w) < 1e-11


@pytest.mark.parametrize("k", [2, 3])
def test_block_operator_matches_global_matrix(k):
    m = Mesh(3, 1, 4)
    A = assemble(m, k)
    x = np.random.default_rng(2).uniform(-1, 1, A.shape[0])
    bo = BlockOperator(m, k)
    assert _rel(bo.apply(x), A @ x) < 1e-14
    cells = [0, 5, 11]
    assert _rel(bo.rows(x, cells), (A @ x).reshape(m.ncells, -1)[cells]) < 1e-14


def test_fast_diagonalization_matches_direct_solve():
    m = Mesh(4, 3, 5)
    A = assemble(m, 2)
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    x = FastDiag(2, 4, 3, 5).solve(b)
    assert _rel(x, spla.spsolve(A.tocsc(), b)) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3])
def test_manufactured_solution_rate(k):
    e = []
    for nc in (8, 16):
        u = FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))
        e.append(l2_error(u, k, nc, nc, nc, sine_exact))
    assert abs(np.log2(e[0] / e[1]) - (k + 1)) < 0.1


def test_discrete_error_below_paper_table3():
    # Table 3 prints the error of an FGMRES solve stopped at 1e-8 with the
    # paper's penalty; the exact discrete solution with that penalty must not
    # be worse. 32^3 cells, extrapolated to 64^3 by the fourth-order rate.
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_table3_l2.txt"))
    paper64 = [r[2] for r in rows if r[0] == 3 and r[1] == 64][0]
    nc = 32
    u = FastDiag(3, nc, nc, nc, pen="paper").solve(rhs_sine(3, nc, nc, nc))
    e32 = l2_error(u, 3, nc, nc, nc, sine_exact)
    assert e32 / 16.0 < paper64
    assert e32 / 16.0 > 0.25 * paper64
