"""Vertex-patch multiplicative Schwarz smoother, in FP64 on the CPU.

Test infrastructure (see ``oracle/__init__``).

What this restates
------------------
* Sec. 7.1 smooths with multiplicative vertex-patch Schwarz (after Cui et al. 2024
  and Witte et al. 2021). A vertex patch is the 2x2x2 block of cells around an
  interior vertex v = (vx, vy, vz) of the mesh, 1 <= v_d <= nc_d - 1: the cells
  v_d - 1 and v_d in each direction d.
* Local solver: exact. A_P = R_P A R_P^T, the restriction of the global SIPG
  matrix to the patch's DoFs, is solved directly (Cholesky of the dense block).
* Multiplicative over colours, additive within one: a patch's colour is the parity
  of its vertex, c = (vx mod 2) + 2 (vy mod 2) + 4 (vz mod 2); two patches of one
  colour share no cell. For each colour in turn r = b - A x is formed and every
  patch P of that colour adds x_P <- x_P + A_P^{-1} r_P.

Readings (the paper cites the smoother without its sweep order): one sweep over
the eight colours per smoothing step, ascending colours when pre-smoothing and
descending when post-smoothing. Every direction needs at least two cells.

Pins (tests/test_oracle_schwarz.py): on a mesh with two cells per direction the
single patch is the whole mesh and one step solves A x = b exactly; on three
cells per direction every colour has one patch, after whose update the residual
vanishes on that patch's DoFs; the patches of a colour are disjoint and together
the colours cover every DoF; the patch DoF lists against a brute-force search by
cell coordinates; the local matrix against the Kronecker sum of Eq. (9) with
the 1D factors restricted to the patch's two cells.
"""
import numpy as np
import scipy.linalg as sla


def patch_vertices(dims):
    """{colour: [(vx, vy, vz), ...]} for the interior vertices of an nx*ny*nz mesh."""
    nx, ny, nz = dims
    if min(dims) < 2:
        raise ValueError("vertex patches need at least two cells per direction")
    out = {c: [] for c in range(8)}
    for vz in range(1, nz):
        for vy in range(1, ny):
            for vx in range(1, nx):
                out[(vx % 2) + 2 * (vy % 2) + 4 * (vz % 2)].append((vx, vy, vz))
    return out


def patch_dofs(k, dims, v):
    """Cell-major DoF indices of the patch around vertex v, listed in the patch's own
    lexicographic order: (Z * 2n + Y) * 2n + X with X = local cell x * n + i (x fastest)."""
    n = k + 1
    nx, ny, _ = dims
    m = 2 * n
    Z, Y, X = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    cx, cy, cz = v[0] - 1 + X // n, v[1] - 1 + Y // n, v[2] - 1 + Z // n
    cell = (cz * ny + cy) * nx + cx
    node = ((Z % n) * n + Y % n) * n + X % n
    return (cell * n ** 3 + node).reshape(-1)


class VertexPatchSmoother:
    """x <- S(x, b) for the global SIPG matrix A (scipy sparse or dense) of degree k on `dims`."""

    def __init__(self, A, k, dims):
        self.A, self.k, self.dims = A, k, dims
        self.colours = patch_vertices(dims)
        self.patches = {}
        for c, verts in self.colours.items():
            lst = []
            for v in verts:
                idx = patch_dofs(k, dims, v)
                AP = A[idx][:, idx]
                AP = AP.toarray() if hasattr(AP, "toarray") else np.asarray(AP)
                lst.append((idx, sla.cho_factor(AP)))
            self.patches[c] = lst

    def colour_step(self, c, x, b):
        """One colour: r = b - A x, then x_P += A_P^{-1} r_P for its patches (in place on a copy)."""
        if not self.patches[c]:
            return x
        r = b - self.A @ x
        x = x.copy()
        for idx, fac in self.patches[c]:
            x[idx] += sla.cho_solve(fac, r[idx])
        return x

    def smooth(self, x, b, reverse=False):
        order = range(7, -1, -1) if reverse else range(8)
        for c in order:
            x = self.colour_step(c, x, b)
        return x
