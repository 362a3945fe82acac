"""Pins of oracle/schwarz.py (vertex-patch multiplicative Schwarz) against facts that do not
depend on it: an exact solve where one patch is the whole mesh, a vanishing patch residual
where a colour has one patch, the Kronecker sum of Eq. (9), and brute-force index searches."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.schwarz import VertexPatchSmoother, patch_dofs, patch_vertices
from oracle.sipg import Mesh, assemble, global_1d


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("k,dims,v", [(1, (3, 4, 2), (2, 1, 1)), (2, (2, 3, 3), (1, 2, 2))])
def test_patch_dofs_against_search_by_coordinates(k, dims, v):
    # decode every global index into (cell coordinates, node) and keep those inside the patch,
    # ordered by the patch's own (Z, Y, X) coordinates
    n = k + 1
    nx, ny, nz = dims
    found = []
    for g in range(nx * ny * nz * n ** 3):
        cell, node = divmod(g, n ** 3)
        cx, cy, cz = cell % nx, (cell // nx) % ny, cell // (nx * ny)
        i, j, l = node % n, (node // n) % n, node // (n * n)
        lx, ly, lz = cx - (v[0] - 1), cy - (v[1] - 1), cz - (v[2] - 1)
        if 0 <= lx < 2 and 0 <= ly < 2 and 0 <= lz < 2:
            X, Y, Z = lx * n + i, ly * n + j, lz * n + l
            found.append(((Z * 2 * n + Y) * 2 * n + X, g))
    expect = [g for _, g in sorted(found)]
    assert list(patch_dofs(k, dims, v)) == expect


def test_colours_are_disjoint_and_cover_every_dof():
    k, dims = 1, (4, 5, 3)
    ndofs = int(np.prod(dims)) * (k + 1) ** 3
    cover = np.zeros(ndofs, dtype=int)
    for c, verts in patch_vertices(dims).items():
        seen = np.zeros(ndofs, dtype=int)
        for v in verts:
            seen[patch_dofs(k, dims, v)] += 1
        assert seen.max() <= 1  # patches of one colour share no DoF
        cover += seen
    assert cover.min() >= 1


@pytest.mark.parametrize("k", [1, 2, 3])
def test_single_patch_mesh_is_solved_exactly(k):
    # 2 x 2 x 2 cells: one interior vertex, its patch is the whole mesh, A_P = A
    dims = (2, 2, 2)
    A = assemble(Mesh(*dims), k)
    b = np.random.default_rng(k).uniform(-1, 1, A.shape[0])
    x = VertexPatchSmoother(A, k, dims).smooth(np.zeros_like(b), b)
    assert _rel(x, spla.spsolve(A.tocsc(), b)) < 1e-12


def test_single_patch_exact_on_anisotropic_box_with_paper_penalty():
    dims, lengths, k = (2, 2, 2), (0.7, 1.3, 0.45), 2
    A = assemble(Mesh(*dims, *lengths), k, "paper")
    b = np.random.default_rng(4).uniform(-1, 1, A.shape[0])
    x = VertexPatchSmoother(A, k, dims).smooth(np.random.default_rng(5).uniform(-1, 1, A.shape[0]), b)
    assert _rel(x, spla.spsolve(A.tocsc(), b)) < 1e-12


def test_patch_residual_vanishes_after_its_colour():
    # 3 x 3 x 3 cells: interior vertices 1, 2 per direction, so every colour holds one patch;
    # after that colour's update the residual is zero on the patch's DoFs
    k, dims = 1, (3, 3, 3)
    A = assemble(Mesh(*dims), k)
    rng = np.random.default_rng(5)
    b, x = rng.uniform(-1, 1, (2, A.shape[0]))
    S = VertexPatchSmoother(A, k, dims)
    for c in range(8):
        (v,) = S.colours[c]
        x = S.colour_step(c, x, b)
        idx = patch_dofs(k, dims, v)
        r = b - A @ x
        assert np.abs(r[idx]).max() < 1e-12 * np.abs(b).max() * 1e3


@pytest.mark.parametrize("k,dims,v", [(1, (4, 3, 2), (1, 2, 1)), (2, (3, 3, 4), (2, 1, 3))])
def test_patch_matrix_is_kronecker_sum_of_restricted_1d_factors(k, dims, v):
    # R_P A R_P^T = L_z[P] (x) M_y[P] (x) M_x[P] + ... with each global 1D factor restricted to the
    # patch's two cells (Eq. (9)); the fast-diagonalization local solver relies on this
    n = k + 1
    A = assemble(Mesh(*dims), k)
    idx = patch_dofs(k, dims, v)
    AP = A[idx][:, idx].toarray()
    f = []
    for d in range(3):
        M, L = global_1d(k, dims[d])
        s = slice((v[d] - 1) * n, (v[d] + 1) * n)
        f.append((M[s, s], L[s, s]))
    (Mx, Lx), (My, Ly), (Mz, Lz) = f
    K = lambda a, b, c: np.kron(a, np.kron(b, c))
    assert _rel(AP, K(Lz, My, Mx) + K(Mz, Ly, Mx) + K(Mz, My, Lx)) < 1e-14


@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
def test_interior_patch_factors_split_into_even_and_odd_eigenproblems(k):
    """A patch around an interior vertex (both neighbouring cells away from the boundary) has 1D
    factors that are mirror-symmetric about the vertex, so its generalized eigenvectors are even or
    odd and the two half-size problems in the even and odd subspaces give the whole spectrum. The
    patches next to the boundary are not symmetric (the boundary face terms). Checked against the
    library's dense generalized eigensolver."""
    import scipy.linalg as sla
    n, P = k + 1, 2 * (k + 1)
    H = P // 2
    J = np.eye(P)[::-1]
    M, L = global_1d(k, 6, pen="config")
    for v, interior in ((1, False), (2, True), (3, True), (5, False)):
        s = slice((v - 1) * n, (v + 1) * n)
        Mp, Lp = M[s, s], L[s, s]
        sym = max(_rel(J @ Mp @ J, Mp), _rel(J @ Lp @ J, Lp))
        if not interior:
            assert sym > 1e-3
            continue
        assert sym < 1e-14
        lam_ref = sla.eigh(Lp, Mp, eigvals_only=True)
        lam, vecs = [], []
        for sg in (1.0, -1.0):
            B = np.zeros((P, H))  # orthonormal basis of the even (sg = 1) or odd subspace
            for m in range(H):
                B[m, m] = B[P - 1 - m, m] = 1.0 / np.sqrt(2.0)
                B[P - 1 - m, m] *= sg
            w, Y = sla.eigh(B.T @ Lp @ B, B.T @ Mp @ B)
            lam += list(w)
            vecs.append(B @ Y)
        V = np.hstack(vecs)
        assert np.allclose(np.sort(lam), lam_ref, rtol=1e-12, atol=0)
        assert _rel(V.T @ Mp @ V, np.eye(P)) < 1e-12
        assert _rel(Lp @ V, Mp @ V @ np.diag(lam)) < 1e-11
        # the parity: even vectors equal their mirror image, odd ones its negative
        assert _rel(J @ vecs[0], vecs[0]) < 1e-14 and _rel(J @ vecs[1], -vecs[1]) < 1e-14


def test_smoother_iteration_contracts_the_energy_error():
    # as a stationary iteration for the SPD SIPG matrix the sweep reduces the A-norm of the error
    k, dims = 1, (4, 4, 4)
    A = assemble(Mesh(*dims), k)
    rng = np.random.default_rng(7)
    xs = rng.uniform(-1, 1, A.shape[0])
    b = A @ xs
    S = VertexPatchSmoother(A, k, dims)
    x = np.zeros_like(b)
    en = lambda e: np.sqrt(e @ (A @ e))
    prev = en(xs - x)
    for it in range(6):
        x = S.smooth(x, b, reverse=bool(it % 2))
        cur = en(xs - x)
        assert cur < 0.9 * prev
        prev = cur


def test_vcycle_with_vertex_patch_smoother_is_exact_on_two_cells():
    # finest 2^3 cells: the pre-smoothing sweep solves exactly (one patch = the mesh), so the
    # coarse correction is zero and the post-smoothing sweep keeps the exact solution
    from oracle.mg import VCycle
    k = 2
    A = assemble(Mesh(2, 2, 2), k)
    b = np.random.default_rng(11).uniform(-1, 1, A.shape[0])
    x = VCycle(k, 2, coarse_nc=1, smoother="vertex_patch")(b)
    assert _rel(x, spla.spsolve(A.tocsc(), b)) < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_vertex_patch_vcycle_preconditions_fgmres_in_few_iterations(k):
    # the property the smoother is chosen for: FGMRES(30) to 1e-10 on the sine problem in at most
    # five iterations (Chebyshev-Jacobi of degree 3 takes 12-14 on the same meshes)
    from oracle.mg import VCycle, fgmres
    from oracle.sipg import BlockOperator
    from oracle.solve import rhs_sine
    nc = 8
    A = BlockOperator(Mesh(nc, nc, nc), k)
    _, its, hist = fgmres(A.apply, VCycle(k, nc, coarse_nc=1, smoother="vertex_patch"), rhs_sine(k, nc, nc, nc))
    assert its <= 5 and hist[-1] <= 1e-10
