"""GPU parity of the patch-wise apply (TP_KERNEL_PATCH: vertex patches of 2x2x2 cells,
Sec. 2.1) against the oracle: the assembled matrix and the oracle's own patch-wise sum
on small meshes (every entry), the block operator on ragged meshes, sampled rows and
the rank-1 closed form of Eq. (9) at full size. Tolerances as for every apply (relative
l2, Sec. 5.2): 1e-12 FP64, 1e-5 FP32."""
import numpy as np
import pytest
import torch

from oracle import patchwise
from oracle.sipg import Mesh, assemble, BlockOperator
from tp_synth import uniform_vector, sample_cells
from tests.gpu_util import TOL, rel_l2, to_device, to_host64
from tests.test_gpu_apply import _rank1_vectors

pytestmark = pytest.mark.gpu

PATCH = 3


def _patch_apply(dims, k, prec, x64, penalty=0, lengths=(1.0, 1.0, 1.0)):
    from paper_2407_09621_gb300 import DGLaplace
    op = DGLaplace(*dims, k, prec, kernel=PATCH, penalty=penalty, lengths=lengths)
    try:
        assert op.info["kernel"] == PATCH and op.info["tensor_path"] == 0 and op.info["tile_cells"] == 8
        assert op.info["flops_per_dof"] == 224 * (k + 1) + 8
        x = to_device(x64, prec)
        y = torch.full_like(x, float("nan"))  # every entry must be written
        op.apply(y, x)
        torch.cuda.synchronize()
        return to_host64(y)
    finally:
        op.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,dims,lengths,pen", [
    (1, (2, 2, 2), (1, 1, 1), 0), (2, (3, 2, 4), (1, 1, 1), 0), (3, (4, 3, 2), (1, 1, 1), 1),
    (2, (5, 3, 2), (0.7, 1.9, 0.45), 0), (4, (2, 3, 2), (1, 1, 1), 0), (5, (3, 2, 2), (1, 1, 1), 0),
    (6, (2, 2, 3), (1, 1, 1), 1), (7, (2, 2, 2), (1, 1, 1), 1)])
def test_patchwise_apply_matches_assembled_matrix(prec, k, dims, lengths, pen):
    A = assemble(Mesh(*dims, *lengths), k, "paper" if pen else "config")
    x = uniform_vector(A.shape[0], seed=40 + k)
    y = _patch_apply(dims, k, prec, x, penalty=pen, lengths=lengths)
    ref = A @ x
    assert rel_l2(y, ref) < TOL[prec]
    if prec == "fp64":
        # the oracle's patch-wise sum: the same patches, the same 1D factors
        y_or = patchwise.apply(x, k, dims, lengths, "paper" if pen else "config")
        assert rel_l2(y, y_or) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,dims", [(3, (9, 6, 11)), (2, (2, 7, 3)), (7, (3, 4, 2)), (1, (16, 2, 5))])
def test_patchwise_apply_ragged_meshes(prec, k, dims):
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=50 + k)
    y = _patch_apply(dims, k, prec, x)
    assert rel_l2(y, BlockOperator(m, k).apply(x)) < TOL[prec]


@pytest.mark.parametrize("k,nc", [(3, 64), (7, 32)])
def test_patchwise_full_size_sampled_and_rank1(k, nc):
    dims = (nc, nc, nc)
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=0)
    y = _patch_apply(dims, k, "fp64", x)
    cells = sample_cells(m.ncells, 1024, seed=3, nx=nc, ny=nc, nz=nc)
    ref = BlockOperator(m, k).rows(x, cells)
    assert rel_l2(y.reshape(m.ncells, -1)[cells], ref) < TOL["fp64"]
    del x, y
    xs, ys = _rank1_vectors(k, nc, seed=23)
    assert rel_l2(_patch_apply(dims, k, "fp64", xs), ys) < TOL["fp64"]


def test_patchwise_host_apply_and_cell_wise_agree():
    """tp_apply_host on a patch-wise operator (no slab pipeline: the patches span slabs) equals its
    tp_apply, and both equal the cell-wise kernel's result to FP64 rounding."""
    from paper_2407_09621_gb300 import DGLaplace
    dims, k = (10, 8, 12), 3
    x64 = uniform_vector(int(np.prod(dims)) * 64, seed=61)
    pw = DGLaplace(*dims, k, "fp64", kernel=PATCH)
    cc = DGLaplace(*dims, k, "fp64", kernel=1)
    try:
        xd = to_device(x64, "fp64")
        yp, yc = torch.empty_like(xd), torch.empty_like(xd)
        pw.apply(yp, xd)
        cc.apply(yc, xd)
        xh = xd.cpu().pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        pw.apply_host(yh, xh)
        torch.cuda.synchronize()
        assert torch.equal(yh, yp.cpu())
        assert rel_l2(to_host64(yp), to_host64(yc)) < 1e-13
    finally:
        pw.close()
        cc.close()


def test_patchwise_is_not_a_multigrid_level_kernel():
    from paper_2407_09621_gb300 import _lib
    mesh = _lib.tp_mesh_create(4, 4, 4)
    op = _lib.tp_dg_laplace_create(mesh, 2, _lib.TP_FP64, kernel=PATCH)
    try:
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_mg_create(op, kernel=PATCH)
        assert e.value.status == _lib.TP_ERR_UNSUPPORTED
        # a patch-wise finest operator is fine: the hierarchy takes only its mesh and degree
        mg = _lib.tp_mg_create(op)
        _lib.tp_mg_destroy(mg)
    finally:
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)
