"""Patch-wise evaluation of the SIPG operator over vertex patches (Sec. 2.1), in FP64.

Test infrastructure (see ``oracle/__init__``).

What this restates
------------------
* Sec. 2.1 evaluates the operator patch by patch: a vertex patch is the 2x2x2
  block of cells around an interior vertex, and on a constant-coefficient
  Cartesian mesh its local operator is the Kronecker sum of Eq. (9),
      A_P = L_z (x) M_y (x) M_x + M_z (x) L_y (x) M_x + M_z (x) M_y (x) L_x,
  with 1D factors of size N = 2(k+1) that hold parts of the cell integrals and
  the face integrals of the patch (the paper's figure of centre, boundary and
  corner patches; the figure itself is not in the text).
* Reading (the split is not printed): in 1D, the patch around interior vertex v
  (1 <= v <= nc - 1) covers cells a = v - 1 and b = v. Every face integral
  belongs to exactly one patch: the interior face at v to the patch around v,
  the boundary face at x = 0 to the patch around v = 1, the one at x = l to the
  patch around v = nc - 1. A cell integral is shared by the patches that hold
  the cell, each taking a weight 1/2 (1 for the first and last cell, which one
  patch holds). So
      M_p = diag(w_a h Mhat, w_b h Mhat),
      L_p = diag(w_a Khat/h, w_b Khat/h) + F_int(v) [+ F_bnd,0 on a if a = 0]
            [+ F_bnd,1 on b if b = nc - 1],
  and the sum over patches of E_v^T M_p E_v is the global 1D mass M and that of
  E_v^T L_p E_v the global 1D SIPG stiffness L. Because the 3D vertex patches
  are the Cartesian products of the 1D ones, the sum over 3D patches of
  E_P^T A_P E_P factors into L_z (x) M_y (x) M_x + ... = A: the patch-wise
  evaluation is the operator itself, evaluated with more work (every cell sits in
  up to eight patches, so each DoF is computed about eight times).
* Every direction needs at least two cells.

Pins (tests/test_oracle_patchwise.py): the 1D sums reproduce ``sipg.global_1d``
(both penalties, nc = 2 .. 5); ``apply`` equals the assembled matrix of
``sipg.assemble`` (itself pinned to brute-force quadrature) on cubic,
non-cubic and anisotropic meshes, k = 1..4 and 7, both penalties.
"""
import numpy as np

from .sipg import Ref1D, penalty, interior_face_1d, boundary_face_1d
from .schwarz import patch_vertices, patch_dofs


def patch_1d(k, nc, v, length=1.0, pen="config"):
    """(M_p, L_p), each 2n x 2n, of the 1D patch around vertex v (1 <= v <= nc - 1)."""
    if not 1 <= v <= nc - 1:
        raise ValueError("v must be an interior vertex")
    ref = Ref1D(k)
    n = ref.n
    h = length / nc
    g = penalty(k, h, pen)
    wa = 1.0 if v - 1 == 0 else 0.5
    wb = 1.0 if v == nc - 1 else 0.5
    M = np.zeros((2 * n, 2 * n))
    L = np.zeros((2 * n, 2 * n))
    a, b = slice(0, n), slice(n, 2 * n)
    M[a, a] = wa * h * ref.Mhat
    M[b, b] = wb * h * ref.Mhat
    L[a, a] = wa * ref.Khat / h
    L[b, b] = wb * ref.Khat / h
    L += interior_face_1d(ref, h, g)
    if v - 1 == 0:
        L[a, a] += boundary_face_1d(ref, h, g, 0)
    if v == nc - 1:
        L[b, b] += boundary_face_1d(ref, h, g, 1)
    return M, L


def sum_1d(k, nc, length=1.0, pen="config"):
    """Sum over the 1D patches of E_v^T M_p E_v and E_v^T L_p E_v (dense nc*n square)."""
    n = k + 1
    M = np.zeros((nc * n, nc * n))
    L = np.zeros((nc * n, nc * n))
    for v in range(1, nc):
        Mp, Lp = patch_1d(k, nc, v, length, pen)
        s = slice((v - 1) * n, (v + 1) * n)
        M[s, s] += Mp
        L[s, s] += Lp
    return M, L


def _kron3_apply(Az, Ay, Ax, u):
    """(Az (x) Ay (x) Ax) u for a patch tensor u[z, y, x]."""
    return np.einsum("ia,jb,kc,abc->ijk", Az, Ay, Ax, u, optimize=True)


def apply(x, k, dims, lengths=(1.0, 1.0, 1.0), pen="config"):
    """y = sum over vertex patches P of E_P^T A_P E_P x (cell-major vectors)."""
    n = k + 1
    m = 2 * n
    if min(dims) < 2:
        raise ValueError("the patch-wise operator needs at least two cells per direction")
    fac = [{v: patch_1d(k, dims[d], v, lengths[d], pen) for v in range(1, dims[d])} for d in range(3)]
    y = np.zeros_like(x, dtype=np.float64)
    for col in range(8):
        for v in patch_vertices(dims)[col]:
            idx = patch_dofs(k, dims, v)
            u = x[idx].reshape(m, m, m)
            (Mx, Lx), (My, Ly), (Mz, Lz) = fac[0][v[0]], fac[1][v[1]], fac[2][v[2]]
            yp = _kron3_apply(Lz, My, Mx, u) + _kron3_apply(Mz, Ly, Mx, u) + _kron3_apply(Mz, My, Lx, u)
            y[idx] += yp.reshape(-1)
    return y


def flops_per_dof(k):
    """Algorithmic flops per DoF of the GPU patch-wise apply: per patch seven contractions of
    (2n)^2 lines with 2n x 2n matrices (a = M_x u, b = L_x u; M_y a, L_y a, M_y b; L_z (M_y a)
    + M_z (L_y a + M_y b)) and one addition per patch DoF, 8 n^3 patch DoFs per cell:
    (7 * 2 * (2n)^4 + (2n)^3) / n^3 = 224 n + 8 (FMA = 2 flops); the paper's N is 2n."""
    n = k + 1
    return 224.0 * n + 8.0
