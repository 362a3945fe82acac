"""Brute-force 3D quadrature assembly of the SIPG form on tiny meshes.

Test infrastructure (see ``oracle/__init__``).

Sec. 2, Eq. (2), evaluated literally: 3D basis functions are evaluated at
physical quadrature points, gradients are 3-vectors, every face carries an
explicit outward normal, jumps are [[v]] = v+ n+ + v- n- (v n on the
boundary) and averages {grad v} are one half of the two traces (the single
trace on the boundary). Nothing here uses the 1D Kronecker factorization of
Eq. (9); this is what pins ``sipg.assemble``. Dense output, so only for a
handful of cells.
"""
import numpy as np

from .basis import gauss_lobatto_nodes, gauss_legendre, lagrange_values, lagrange_derivatives
from .sipg import penalty


def _cell_origin(mesh, c):
    cx, cy, cz = mesh.coords(c)
    return np.array([cx * mesh.h[0], cy * mesh.h[1], cz * mesh.h[2]])


def phys_basis(mesh, k, c, pts):
    """Values (P, n^3) and gradients (P, n^3, 3) of cell c's basis at points (P, 3).

    phi_(l,j,i)(x) = phi_i(xi_0) phi_j(xi_1) phi_l(xi_2), xi = (x - x_c) / h.
    """
    nodes = gauss_lobatto_nodes(k)
    h = np.array(mesh.h)
    xi = (pts - _cell_origin(mesh, c)) / h
    v = [lagrange_values(nodes, xi[:, d]) for d in range(3)]          # (P, n)
    dv = [lagrange_derivatives(nodes, xi[:, d]) / h[d] for d in range(3)]
    val = np.einsum("pl,pj,pi->plji", v[2], v[1], v[0]).reshape(len(pts), -1)
    gx = np.einsum("pl,pj,pi->plji", v[2], v[1], dv[0]).reshape(len(pts), -1)
    gy = np.einsum("pl,pj,pi->plji", v[2], dv[1], v[0]).reshape(len(pts), -1)
    gz = np.einsum("pl,pj,pi->plji", dv[2], v[1], v[0]).reshape(len(pts), -1)
    return val, np.stack([gx, gy, gz], axis=-1)


def assemble_dense(mesh, k, pen="config", q=None):
    """Dense SIPG matrix (row = test, column = trial), cell-major layout."""
    n = k + 1
    nb = n ** 3
    q = q or k + 2
    xq, wq = gauss_legendre(q)
    N = mesh.ncells * nb
    A = np.zeros((N, N))
    h = np.array(mesh.h)
    # volume terms: int_K grad phi_b . grad phi_a
    for c in range(mesh.ncells):
        g = np.stack(np.meshgrid(xq, xq, xq, indexing="ij"), -1).reshape(-1, 3)
        w = np.einsum("a,b,c->abc", wq, wq, wq).reshape(-1) * np.prod(h)
        pts = _cell_origin(mesh, c) + g * h
        _, grad = phys_basis(mesh, k, c, pts)
        s = slice(c * nb, (c + 1) * nb)
        A[s, s] += np.einsum("p,pad,pbd->ab", w, grad, grad)
    # face terms
    for c in range(mesh.ncells):
        co = mesh.coords(c)
        for d in range(3):
            for side in (0, 1):
                t = [e for e in range(3) if e != d]
                g2 = np.stack(np.meshgrid(xq, xq, indexing="ij"), -1).reshape(-1, 2)
                w = np.einsum("a,b->ab", wq, wq).reshape(-1) * h[t[0]] * h[t[1]]
                pts = np.zeros((len(g2), 3))
                o = _cell_origin(mesh, c)
                pts[:, t[0]] = o[t[0]] + g2[:, 0] * h[t[0]]
                pts[:, t[1]] = o[t[1]] + g2[:, 1] * h[t[1]]
                pts[:, d] = o[d] + side * h[d]
                normal = np.zeros(3)
                normal[d] = 1.0 if side == 1 else -1.0
                co2 = list(co)
                co2[d] += 1 if side == 1 else -1
                interior = 0 <= co2[d] < mesh.nc[d]
                if interior and side == 0:
                    continue  # each interior face once, from its low cell
                gam = penalty(k, h[d], pen)
                cells = [c]
                normals = [normal]
                if interior:
                    cells.append(mesh.cell(*co2))
                    normals.append(-normal)
                vals, grads, jumps = [], [], []
                for cc, nn in zip(cells, normals):
                    v, gr = phys_basis(mesh, k, cc, pts)
                    vals.append(v)
                    grads.append(gr)
                    jumps.append(v[:, :, None] * nn[None, None, :])   # [[phi]] part, (P, nb, 3)
                fac = 0.5 if interior else 1.0
                J = np.concatenate(jumps, axis=1)                      # (P, m, 3)
                Avg = fac * np.concatenate(grads, axis=1)              # (P, m, 3)
                blk = (gam * np.einsum("p,pad,pbd->ab", w, J, J)
                       - np.einsum("p,pad,pbd->ab", w, J, Avg)        # -{grad u}.[[v]]: a test, b trial
                       - np.einsum("p,pad,pbd->ab", w, Avg, J))       # -[[u]].{grad v}
                idx = np.concatenate([np.arange(cc * nb, (cc + 1) * nb) for cc in cells])
                A[np.ix_(idx, idx)] += blk
    return A
