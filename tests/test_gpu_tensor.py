"""GPU parity of the tensor-core apply (mma.sync, FP16/BF16 operands, FP32
accumulation) and of its Algorithm 1 error-corrected variant, against the FP64
oracle; and the multigrid preconditioner running on it.

Tolerances (relative l2, Sec. 5.2): FP16/BF16 vectors 5e-3; FP32 vectors with
FP16 operands and error correction 1e-5 (Algorithm 1 recovers single
precision: the dropped da*db term is 2^-22 relative); with BF16 operands the
split keeps 16 bits, so 1e-4; without correction the operand rounding alone
allows 5e-3."""
import numpy as np
import pytest
import torch

from oracle.sipg import Mesh, BlockOperator
from oracle.mg import VCycle
from oracle.solve import FastDiag, rhs_sine, l2_error, sine_exact
from tp_synth import uniform_vector
from tests.gpu_util import rel_l2, to_device, to_host64

pytestmark = pytest.mark.gpu

TP_FP32, TP_FP16, TP_BF16, TENSOR = 1, 2, 3, 2


def _apply_tc(dims, k, prec, x64, ec=0, tc_type=TP_FP16):
    from paper_2407_09621_gb300 import DGLaplace
    op = DGLaplace(*dims, k, prec, kernel=TENSOR, ec=ec, tc_type=tc_type)
    try:
        assert op.info["kernel"] == TENSOR
        x = to_device(x64, prec)
        y = torch.empty_like(x)
        op.apply(y, x)
        op.check()
        return to_host64(y)
    finally:
        op.close()


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("prec,ec", [("fp16", 0), ("bf16", 0), ("fp16", 1), ("bf16", 1)])
@pytest.mark.parametrize("dims", [(5, 3, 4), (1, 1, 1), (67, 2, 1), (3, 1, 70)])
def test_half_storage_tensor_apply(k, prec, ec, dims):
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=20 + k)
    y = _apply_tc(dims, k, prec, x, ec=ec)
    assert rel_l2(y, BlockOperator(m, k).apply(x)) < 5e-3


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("tc_type,ec,tol", [(TP_FP16, 1, 1e-5), (TP_BF16, 1, 1e-4), (TP_FP16, 0, 5e-3),
                                            (TP_BF16, 0, 2e-2)])
def test_fp32_storage_tensor_apply(k, tc_type, ec, tol):
    dims = (6, 5, 7)
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=30 + k)
    y = _apply_tc(dims, k, "fp32", x, ec=ec, tc_type=tc_type)
    assert rel_l2(y, BlockOperator(m, k).apply(x)) < tol


def test_error_correction_improves_accuracy():
    dims, k = (8, 8, 8), 3
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * 64, seed=5)
    ref = BlockOperator(m, k).apply(x)
    e_plain = rel_l2(_apply_tc(dims, k, "fp32", x, ec=0), ref)
    e_ec = rel_l2(_apply_tc(dims, k, "fp32", x, ec=1), ref)
    assert e_ec < 1e-2 * e_plain


@pytest.mark.parametrize("k,nc", [(3, 80), (2, 107)])
def test_config2_tensor_sampled(k, nc):
    from tp_synth import sample_cells
    m = Mesh(nc, nc, nc)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=0)
    cells = sample_cells(m.ncells, 512, seed=2, nx=nc, ny=nc, nz=nc)
    ref = BlockOperator(m, k).rows(x, cells)
    for prec in ("fp16", "bf16"):
        y = _apply_tc((nc, nc, nc), k, prec, x)
        assert rel_l2(y.reshape(m.ncells, -1)[cells], ref) < 5e-3


def test_vcycle_on_tensor_kernel_with_error_correction():
    from paper_2407_09621_gb300 import _lib
    k, nc, lmax = 3, 8, 2.9
    mesh = _lib.tp_mesh_create(nc, nc, nc)
    op = _lib.tp_dg_laplace_create(mesh, k, _lib.TP_FP64)
    mg = _lib.tp_mg_create(op, lmax=lmax, coarse_cells=1, precision=_lib.TP_FP32, kernel=TENSOR, ec=1)
    try:
        n = nc ** 3 * 64
        b, x0 = uniform_vector(n, seed=3), uniform_vector(n, seed=4)
        x = torch.from_numpy(x0).float().cuda()
        _lib.tp_vcycle(mg, x.data_ptr(), torch.from_numpy(b).float().cuda().data_ptr())
        torch.cuda.synchronize()
        ref_mg = VCycle(k, nc, coarse_nc=1)
        ref_mg.lmax = [None] + [lmax] * (len(ref_mg.levels) - 1)
        ref = ref_mg.vcycle(len(ref_mg.levels) - 1, b, x0)
        assert rel_l2(x.double().cpu().numpy(), ref) < 1e-4
    finally:
        _lib.tp_mg_destroy(mg)
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)


@pytest.mark.parametrize("ec", [1, 0])
def test_solve_with_tensor_vcycle(ec):
    from paper_2407_09621_gb300 import _lib
    k, nc = 3, 32
    mesh = _lib.tp_mesh_create(nc, nc, nc)
    op = _lib.tp_dg_laplace_create(mesh, k, _lib.TP_FP64)
    mg = _lib.tp_mg_create(op, precision=_lib.TP_FP32, kernel=TENSOR, ec=ec)
    solver = _lib.tp_fgmres_create(op, mg, 30)
    try:
        b = torch.from_numpy(rhs_sine(k, nc, nc, nc)).cuda()
        x = torch.zeros_like(b)
        st, info = _lib.tp_fgmres_solve(solver, x.data_ptr(), b.data_ptr(), 1e-10, 200)
        assert info["converged"] == 1
        u = FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))
        e_mixed = l2_error(x.cpu().numpy(), k, nc, nc, nc, sine_exact)
        e_exact = l2_error(u, k, nc, nc, nc, sine_exact)
        assert abs(e_mixed - e_exact) <= 0.01 * e_exact
    finally:
        _lib.tp_solver_destroy(solver)
        _lib.tp_mg_destroy(mg)
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("dims", [(9, 7, 11), (16, 16, 16), (40, 40, 20), (2, 130, 3)])
def test_tcgen05_apply_tiles(prec, dims):
    """k = 3 with half-precision vectors runs on tcgen05: tiles of 128 cells, a ragged last
    tile (693 cells), exact tiles (4096), more tiles than SMs (250 tiles, persistent loop),
    and a y-stride that is not a multiple of the tile (2 x 130 x 3)."""
    from paper_2407_09621_gb300 import DGLaplace
    op = DGLaplace(*dims, 3, prec, kernel=TENSOR)
    try:
        assert op.info["tensor_path"] == 2
    finally:
        op.close()
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * 64, seed=41)
    y = _apply_tc(dims, 3, prec, x)
    assert rel_l2(y, BlockOperator(m, 3).apply(x)) < 5e-3


@pytest.mark.parametrize("k,prec,path", [(2, "fp16", 1), (3, "fp32", 1), (3, "fp16", 2), (3, "bf16", 2)])
def test_tensor_path_selection(k, prec, path):
    from paper_2407_09621_gb300 import DGLaplace
    op = DGLaplace(3, 3, 3, k, prec, kernel=TENSOR)
    try:
        assert op.info["tensor_path"] == path
    finally:
        op.close()


@pytest.mark.parametrize("tc_type", [TP_FP16, TP_BF16])
def test_error_correction_modes_order_the_errors(tc_type):
    """Refining one operand of the half-precision products (ec = 2: the operator matrices, ec = 3:
    the vector side) removes one of the two rounding contributions; refining both (Algorithm 1,
    ec = 1) removes both."""
    dims, k = (6, 5, 7), 3
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * 64, seed=31)
    ref = BlockOperator(m, k).apply(x)
    err = {ec: rel_l2(_apply_tc(dims, k, "fp32", x, ec=ec, tc_type=tc_type), ref) for ec in (0, 1, 2, 3)}
    assert err[1] < 1e-2 * err[0]
    assert err[2] < err[0] and err[3] < err[0]
    assert err[1] < min(err[2], err[3])
