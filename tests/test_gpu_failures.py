"""Failure detection without a GPU fault: non-finite inputs to the FGMRES solve are
reported as TP_ERR_NONFINITE, a bounded wait of the tcgen05 apply that runs out is
reported as TP_ERR_TIMEOUT by tp_op_check and leaves the context usable, and a solve
reports whether its V-cycle ran as the captured CUDA graph.

The timeout is provoked through include/tp_test.h: the wait limit is shortened to a
few milliseconds and CTA 0 skips the copy of its first input tile, so the barrier of
that slot never completes (no trap, no bad address, no unbounded wait)."""
import numpy as np
import pytest
import torch

from oracle.sipg import Mesh, BlockOperator
from oracle.solve import rhs_sine
from tp_synth import uniform_vector
from tests.gpu_util import rel_l2, to_device, to_host64

pytestmark = pytest.mark.gpu

TENSOR = 2


def _solver(k, nc, with_mg=True):
    from paper_2407_09621_gb300 import _lib
    mesh = _lib.tp_mesh_create(nc, nc, nc)
    op = _lib.tp_dg_laplace_create(mesh, k, _lib.TP_FP64)
    mg = _lib.tp_mg_create(op, precision=_lib.TP_FP32) if with_mg else None
    solver = _lib.tp_fgmres_create(op, mg, 30)

    def close():
        _lib.tp_solver_destroy(solver)
        if mg:
            _lib.tp_mg_destroy(mg)
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)
    return solver, close


@pytest.mark.parametrize("where", ["b_nan", "b_inf", "x0_nan"])
def test_nonfinite_input_is_reported(where):
    from paper_2407_09621_gb300 import _lib
    k, nc = 2, 8
    solver, close = _solver(k, nc)
    try:
        b = torch.from_numpy(rhs_sine(k, nc, nc, nc)).cuda()
        x = torch.zeros_like(b)
        if where == "b_nan":
            b[12345] = float("nan")
        elif where == "b_inf":
            b[7] = float("inf")
        else:
            x[100] = float("nan")
        st, info = _lib.tp_fgmres_solve(solver, x.data_ptr(), b.data_ptr(), 1e-10, 50, raise_on_error=False)
        assert st == _lib.TP_ERR_NONFINITE
        assert "non-finite" in _lib.tp_last_error()
        assert info["converged"] == 0
        # the solver and the context stay usable
        b = torch.from_numpy(rhs_sine(k, nc, nc, nc)).cuda()
        x.zero_()
        st, info = _lib.tp_fgmres_solve(solver, x.data_ptr(), b.data_ptr(), 1e-10, 50, raise_on_error=False)
        assert st == _lib.TP_OK and info["converged"] == 1
    finally:
        close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tcgen05_wait_timeout_is_reported_and_recoverable(prec):
    from paper_2407_09621_gb300 import DGLaplace, TPError, _lib
    dims = (4, 4, 4)  # one tile of 64 cells: one CTA
    m = Mesh(*dims)
    x64 = uniform_vector(m.ncells * 64, seed=9)
    op = DGLaplace(*dims, 3, prec, kernel=TENSOR)
    try:
        assert op.info["tensor_path"] == 2
        x = to_device(x64, prec)
        y = torch.zeros_like(x)
        _lib.tp_test_set_wait_fault(op.op, 1, 0.005)
        op.apply(y, x)
        with pytest.raises(TPError) as e:
            op.check()
        assert e.value.status == _lib.TP_ERR_TIMEOUT
        assert "gave up" in str(e.value)
        # the status word is cleared by the check, the context is intact: a normal launch works
        _lib.tp_test_set_wait_fault(op.op, 0, 0.0)
        op.apply(y, x)
        op.check()
        assert rel_l2(to_host64(y), BlockOperator(m, 3).apply(x64)) < 5e-3
    finally:
        op.close()


def test_wait_fault_hook_validates_its_arguments():
    from paper_2407_09621_gb300 import DGLaplace, TPError, _lib
    cc = DGLaplace(2, 2, 2, 3, "fp16", kernel=1)
    tc = DGLaplace(2, 2, 2, 3, "fp16", kernel=TENSOR)
    try:
        with pytest.raises(TPError) as e:
            _lib.tp_test_set_wait_fault(cc.op, 1, 0.01)
        assert e.value.status == _lib.TP_ERR_UNSUPPORTED
        with pytest.raises(TPError) as e:
            _lib.tp_test_set_wait_fault(tc.op, 0, -1.0)
        assert e.value.status == _lib.TP_ERR_INVALID_ARG
        _lib.tp_test_set_wait_fault(tc.op, 0, 0.0)
    finally:
        cc.close()
        tc.close()


def test_solve_reports_the_captured_vcycle_graph():
    from paper_2407_09621_gb300 import _lib
    k, nc = 2, 16
    b = torch.from_numpy(rhs_sine(k, nc, nc, nc)).cuda()
    for with_mg, expect in ((True, 1), (False, 0)):
        solver, close = _solver(k, nc, with_mg)
        try:
            x = torch.zeros_like(b)
            st, info = _lib.tp_fgmres_solve(solver, x.data_ptr(), b.data_ptr(), 1e-6, 300, raise_on_error=False)
            assert info["vcycle_graph"] == expect
            assert info["iterations"] >= 1
        finally:
            close()
