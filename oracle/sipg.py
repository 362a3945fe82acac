"""SIPG discretization of -Laplace(u) = f on a Cartesian hex mesh: explicit
element and face matrices from 1D matrices by Kronecker products, summed
into a global sparse matrix.

Test infrastructure (see ``oracle/__init__``).

What this restates
------------------
* Sec. 2, Eq. (2): the symmetric interior penalty bilinear form
      a(u, v) = sum_K int_K grad u . grad v
              + sum_e int_e ( g_e [[u]].[[v]] - {grad u}.[[v]] - [[u]].{grad v} ).
  The printed form shows averages {u n} where SIPG has jumps; the brackets
  were lost in conversion (the source loads stmaryrd, the jump-bracket
  package). Reading: [[v]] = v+ n+ + v- n- on interior faces and v n on
  boundary faces; {v} is the average inside and the one-sided trace on the
  boundary (Sec. 2, below Eq. (1)).
* Penalty: Sec. 2 gives g_e = k(k+1)(1/h+ + 1/h-) ("paper"); the default
  here is (k+1)^2/h ("config") on interior and boundary faces. h is the cell
  width normal to the face; on a boundary face h+ = h- = h.
* Sec. 2.1, Eq. (9): on a constant-coefficient Cartesian mesh the operator is
  L_2 (x) M_1 (x) M_0 + M_2 (x) L_1 (x) M_0 + M_2 (x) M_1 (x) L_0. Every
  element and face matrix below is such a Kronecker product of 1D matrices.
* Quadrature: (k+1)-point Gauss-Legendre per direction, exact for the mass
  and stiffness integrands on affine cells (the lumped Gauss-Lobatto
  collocation mass is a different operator and is not used).

Layout: cell-major, g = ((cz*ny + cy)*nx + cx)*n^3 + (l*n + j)*n + i with
n = k+1 and i the x node (fastest).

Pinned by tests/test_oracle_sipg.py: brute-force 3D quadrature of Eq. (2)
on one- and two-cell meshes (oracle/brute.py; k <= 5, 7 and 8), symmetry,
positive definiteness, the hand-derived k = 1 one-cell 1D matrix, the
spectral closed form of Eq. (9), and agreement of the global, block and
Kronecker-sum forms (``kron_apply``, the one used for degrees up to 15).
"""
import numpy as np
import scipy.sparse as sp

from .basis import gauss_lobatto_nodes, gauss_legendre, lagrange_values, lagrange_derivatives


def penalty(k, h, mode="config"):
    """Penalty g_e for a face whose adjacent cells have width h normal to it."""
    if mode == "config":
        return (k + 1) ** 2 / h
    if mode == "paper":  # Sec. 2: k(k+1)(1/h+ + 1/h-)
        return k * (k + 1) * (1.0 / h + 1.0 / h)
    raise ValueError(mode)


class Ref1D:
    """Reference-interval data on [0, 1] for degree k (Sec. 2)."""

    def __init__(self, k):
        self.k = k
        self.n = k + 1
        self.nodes = gauss_lobatto_nodes(k)
        xq, wq = gauss_legendre(k + 1)
        phi = lagrange_values(self.nodes, xq)       # (q, n)
        dphi = lagrange_derivatives(self.nodes, xq)  # (q, n)
        self.Mhat = phi.T @ (wq[:, None] * phi)     # int phi_i phi_j
        self.Khat = dphi.T @ (wq[:, None] * dphi)   # int phi_i' phi_j'
        self.v0 = lagrange_values(self.nodes, [0.0])[0]
        self.v1 = lagrange_values(self.nodes, [1.0])[0]
        self.d0 = lagrange_derivatives(self.nodes, [0.0])[0]
        self.d1 = lagrange_derivatives(self.nodes, [1.0])[0]


def face_matrix(jump, avg, gamma):
    """Face integrand of Eq. (2) for basis vectors: row = test, column = trial.

    jump[a] = [[phi_a]] . n_e, avg[a] = {d phi_a / d n_e} for every basis
    function a touching the face; the entry (a, b) is
    g [[phi_b]][[phi_a]] - {phi_b'}[[phi_a]] - [[phi_b]]{phi_a'}.
    """
    return gamma * np.outer(jump, jump) - np.outer(jump, avg) - np.outer(avg, jump)


def interior_face_1d(ref, h, gamma):
    """2n x 2n face matrix between a left cell (first n) and a right cell.

    With n_e = +x: [[u]] = u_L - u_R, {u'} = (u_L' + u_R') / 2.
    """
    jump = np.concatenate([ref.v1, -ref.v0])
    avg = 0.5 * np.concatenate([ref.d1, ref.d0]) / h
    return face_matrix(jump, avg, gamma)


def boundary_face_1d(ref, h, gamma, side):
    """n x n boundary face matrix; side 0 is the low end (n = -1), 1 the high end."""
    if side == 0:
        return face_matrix(-ref.v0, ref.d0 / h, gamma)
    return face_matrix(ref.v1, ref.d1 / h, gamma)


def global_1d(k, nc, length=1.0, pen="config"):
    """Global 1D DG mass M and SIPG stiffness L on nc cells (dense, nc*n square).

    M is block diagonal with h*Mhat; L = blockdiag(Khat/h) + all face matrices.
    These are the 1D factors of Eq. (9).
    """
    ref = Ref1D(k)
    n = ref.n
    h = length / nc
    g = penalty(k, h, pen)
    N = nc * n
    M = np.zeros((N, N))
    L = np.zeros((N, N))
    for c in range(nc):
        s = slice(c * n, (c + 1) * n)
        M[s, s] += h * ref.Mhat
        L[s, s] += ref.Khat / h
    for c in range(nc - 1):
        s = slice(c * n, (c + 2) * n)
        L[s, s] += interior_face_1d(ref, h, g)
    L[0:n, 0:n] += boundary_face_1d(ref, h, g, 0)
    L[N - n:N, N - n:N] += boundary_face_1d(ref, h, g, 1)
    return M, L


class Mesh:
    """Uniform Cartesian mesh of [0,lx]x[0,ly]x[0,lz] with nx*ny*nz cells."""

    def __init__(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0):
        self.nc = (nx, ny, nz)
        self.h = (lx / nx, ly / ny, lz / nz)
        self.length = (lx, ly, lz)

    @property
    def ncells(self):
        return self.nc[0] * self.nc[1] * self.nc[2]

    def cell(self, cx, cy, cz):
        nx, ny, _ = self.nc
        return (cz * ny + cy) * nx + cx

    def coords(self, c):
        nx, ny, _ = self.nc
        return c % nx, (c // nx) % ny, c // (nx * ny)


def _kron3(az, ay, ax):
    """az (x) ay (x) ax with the x index fastest."""
    return np.kron(az, np.kron(ay, ax))


def _place(d, blk, Mx, My, Mz):
    """Tangential Kronecker placement of a 1D normal-direction block."""
    if d == 0:
        return _kron3(Mz, My, blk)
    if d == 1:
        return _kron3(Mz, blk, Mx)
    return _kron3(blk, My, Mx)


def assemble(mesh, k, pen="config"):
    """Global SIPG matrix, cell-major layout, by an element loop plus a face loop.

    Sec. 2.1 steps (ii)(b)-(c): every cell contributes its element stiffness
    K_z(x)M_y(x)M_x + M_z(x)K_y(x)M_x + M_z(x)M_y(x)K_x, every face its face
    matrix (normal-direction 1D face matrix (x) tangential 1D masses); the
    sums are accumulated block-wise and returned as scipy CSR.
    """
    ref = Ref1D(k)
    n = ref.n
    nx, ny, nz = mesh.nc
    hx, hy, hz = mesh.h
    Ms = [h * ref.Mhat for h in mesh.h]
    Ks = [ref.Khat / h for h in mesh.h]
    Mx, My, Mz = Ms
    el = _kron3(Mz, My, Ks[0]) + _kron3(Mz, Ks[1], Mx) + _kron3(Ks[2], My, Mx)
    blocks = {}

    def add(r, c, b):
        if (r, c) in blocks:
            blocks[(r, c)] = blocks[(r, c)] + b
        else:
            blocks[(r, c)] = b.copy()

    for c in range(mesh.ncells):
        add(c, c, el)
    for d in range(3):
        h = mesh.h[d]
        g = penalty(k, h, pen)
        Fi = interior_face_1d(ref, h, g)
        Fb = [boundary_face_1d(ref, h, g, s) for s in (0, 1)]
        for c in range(mesh.ncells):
            co = list(mesh.coords(c))
            if co[d] == 0:
                add(c, c, _place(d, Fb[0], Mx, My, Mz))
            if co[d] == mesh.nc[d] - 1:
                add(c, c, _place(d, Fb[1], Mx, My, Mz))
            else:
                co2 = list(co)
                co2[d] += 1
                cr = mesh.cell(*co2)
                add(c, c, _place(d, Fi[:n, :n], Mx, My, Mz))
                add(c, cr, _place(d, Fi[:n, n:], Mx, My, Mz))
                add(cr, c, _place(d, Fi[n:, :n], Mx, My, Mz))
                add(cr, cr, _place(d, Fi[n:, n:], Mx, My, Mz))
    keys = sorted(blocks)
    nb = n ** 3
    indptr = np.zeros(mesh.ncells + 1, dtype=np.int64)
    for r, _ in keys:
        indptr[r + 1] += 1
    indptr = np.cumsum(indptr)
    indices = np.array([c for _, c in keys], dtype=np.int64)
    data = np.stack([blocks[kk] for kk in keys])
    A = sp.bsr_matrix((data, indices, indptr), shape=(mesh.ncells * nb, mesh.ncells * nb))
    return A.tocsr()


class BlockOperator:
    """y = A x evaluated block-row by block-row without a global matrix.

    Same element and face matrices as ``assemble``; since the mesh is uniform,
    the diagonal block of a cell depends only on which of its faces lie on the
    boundary, and the off-diagonal block only on the face direction and side.
    y_c = A_cc x_c + sum over the (up to) six face neighbours A_c,nb x_nb.
    Used for meshes too large to assemble and for sampled rows at full size.
    """

    def __init__(self, mesh, k, pen="config"):
        ref = Ref1D(k)
        self.mesh, self.k, self.n = mesh, k, ref.n
        n = ref.n
        Ms = [h * ref.Mhat for h in mesh.h]
        Ks = [ref.Khat / h for h in mesh.h]
        Mx, My, Mz = Ms
        el = _kron3(Mz, My, Ks[0]) + _kron3(Mz, Ks[1], Mx) + _kron3(Ks[2], My, Mx)
        # per direction: diagonal face contribution for (low face status, high face status)
        diag_parts = []
        self.off = {}
        for d in range(3):
            h = mesh.h[d]
            g = penalty(k, h, pen)
            Fi = interior_face_1d(ref, h, g)
            Fb = [boundary_face_1d(ref, h, g, s) for s in (0, 1)]
            low = {True: Fb[0], False: Fi[n:, n:]}   # face at the low end: boundary or interior (cell is "right")
            high = {True: Fb[1], False: Fi[:n, :n]}  # face at the high end
            parts = {}
            for lb in (False, True):
                for hb in (False, True):
                    parts[(lb, hb)] = _place(d, low[lb] + high[hb], Mx, My, Mz)
            diag_parts.append(parts)
            self.off[(d, -1)] = _place(d, Fi[n:, :n], Mx, My, Mz)  # row cell's low neighbour
            self.off[(d, +1)] = _place(d, Fi[:n, n:], Mx, My, Mz)  # row cell's high neighbour
        self.diag = {}
        for key in [(a, b, c, d, e, f) for a in (0, 1) for b in (0, 1) for c in (0, 1)
                    for d in (0, 1) for e in (0, 1) for f in (0, 1)]:
            blk = el.copy()
            for dd in range(3):
                blk = blk + diag_parts[dd][(bool(key[2 * dd]), bool(key[2 * dd + 1]))]
            self.diag[key] = blk

    def _diag_key(self, co):
        key = []
        for d in range(3):
            key += [co[d] == 0, co[d] == self.mesh.nc[d] - 1]
        return tuple(int(b) for b in key)

    def rows(self, x, cells):
        """y restricted to the given cells: array (len(cells), n^3)."""
        mesh, nb = self.mesh, self.n ** 3
        X = np.asarray(x, dtype=np.float64).reshape(mesh.ncells, nb)
        out = np.zeros((len(cells), nb))
        for r, c in enumerate(cells):
            co = mesh.coords(int(c))
            y = self.diag[self._diag_key(co)] @ X[c]
            for d in range(3):
                for s in (-1, 1):
                    co2 = list(co)
                    co2[d] += s
                    if 0 <= co2[d] < mesh.nc[d]:
                        y = y + self.off[(d, s)] @ X[mesh.cell(*co2)]
            out[r] = y
        return out

    def apply(self, x):
        """Full y = A x (batched over cells of equal block type)."""
        mesh, nb = self.mesh, self.n ** 3
        nx, ny, nz = mesh.nc
        X = np.asarray(x, dtype=np.float64).reshape(nz, ny, nx, nb)
        Y = np.zeros_like(X)
        cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        co = (cx, cy, cz)
        flags = []
        for d in range(3):
            flags += [co[d] == 0, co[d] == mesh.nc[d] - 1]
        code = np.zeros(X.shape[:3], dtype=np.int64)
        for b, f in enumerate(flags):
            code |= f.astype(np.int64) << b
        for key, blk in self.diag.items():
            kc = sum(v << b for b, v in enumerate(key))
            sel = code == kc
            if sel.any():
                Y[sel] += X[sel] @ blk.T
        # off-diagonal: neighbour along axis d (array axis 2 - d)
        for d in range(3):
            ax = 2 - d
            B_lo, B_hi = self.off[(d, -1)], self.off[(d, +1)]
            m = X.shape[ax]
            if m > 1:
                lo = [slice(None)] * 3
                hi = [slice(None)] * 3
                lo[ax] = slice(1, m)      # cells that have a low neighbour
                hi[ax] = slice(0, m - 1)  # their low neighbours
                Y[tuple(lo)] += X[tuple(hi)] @ B_lo.T
                Y[tuple(hi)] += X[tuple(lo)] @ B_hi.T
        return Y.reshape(-1)


def lex_to_cell_major(k, nx, ny, nz):
    """perm with v_cell[g] = v_lex[perm[g]] for the cell-major layout.

    Lexicographic global-node order: ((gz*(ny*n) + gy)*(nx*n) + gx) with
    gx = cx*n + i; this is the index order of kron(Lz, kron(Ly, Lx)) built
    from global 1D matrices.
    """
    n = k + 1
    cz, cy, cx, l, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                                      np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    gx, gy, gz = cx * n + i, cy * n + j, cz * n + l
    return ((gz * (ny * n) + gy) * (nx * n) + gx).reshape(-1)


def kron_apply(x, k, dims, lengths=(1.0, 1.0, 1.0), pen="config"):
    """y = A x by the Kronecker-sum form of Eq. (9) with each direction's global 1D factors:
    A = L_z (x) M_y (x) M_x + M_z (x) L_y (x) M_x + M_z (x) M_y (x) L_x in the lexicographic
    global-node order, x and y in the cell-major layout. The 1D factors are dense (nc*n
    square), so this serves meshes of a few cells per direction at any degree."""
    nx, ny, nz = dims
    n = k + 1
    (Mx, Lx), (My, Ly), (Mz, Lz) = [global_1d(k, nc, length=ln, pen=pen) for nc, ln in zip(dims, lengths)]
    perm = lex_to_cell_major(k, nx, ny, nz)
    x_lex = np.empty(len(perm))
    x_lex[perm] = np.asarray(x, dtype=np.float64)
    X = x_lex.reshape(nz * n, ny * n, nx * n)
    Y = (np.einsum("zc,yb,xa,cba->zyx", Lz, My, Mx, X, optimize=True)
         + np.einsum("zc,yb,xa,cba->zyx", Mz, Ly, Mx, X, optimize=True)
         + np.einsum("zc,yb,xa,cba->zyx", Mz, My, Lx, X, optimize=True))
    return Y.reshape(-1)[perm]
