"""Batched uneven Poisson solves (concurrent streams, graph-captured V-cycles)
against the oracle: every problem's solution vs its exact discrete solution by
fast diagonalization, its L2 error vs the oracle's, and the concurrent run vs
the one-stream run of the same batch."""
import numpy as np
import pytest
import torch

from oracle.solve import FastDiag, rhs_modes, l2_error
from tp_synth import batch_problems
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


def _exact(modes):
    return lambda X, Y, Z: sum(a * np.sin(p * np.pi * X) * np.sin(q * np.pi * Y) * np.sin(r * np.pi * Z)
                               for a, p, q, r in modes)


@pytest.mark.parametrize("autotune,smoother", [(0, 0), (1, 0), (0, 1)])
def test_small_uneven_batch_matches_oracle(autotune, smoother):
    from paper_2407_09621_gb300 import _lib
    probs = batch_problems(count=6, seed_base=2000, cells_choices=(4, 6, 8), degrees=(1, 2, 3, 4, 5, 6, 7))
    xs = []
    for p in probs:
        xs.append(torch.zeros(p["dofs"], dtype=torch.float64, device="cuda"))
        p["x_ptr"] = xs[-1].data_ptr()
    res, total = _lib.tp_batch_solve(probs, streams=4, autotune=autotune, smoother=smoother)
    assert total > 0
    for p, r, x in zip(probs, res, xs):
        c, k = p["cells"], p["k"]
        assert r["converged"] == 1 and r["status"] == 0
        u = FastDiag(k, c, c, c).solve(rhs_modes(k, c, c, c, p["modes"]))
        assert rel_l2(x.cpu().numpy(), u) < 1e-7
        e_ref = l2_error(u, k, c, c, c, _exact(p["modes"]))
        if e_ref > 1e-10:
            assert abs(r["l2_error"] - e_ref) <= 0.01 * e_ref
        else:
            assert r["l2_error"] <= max(1.01 * e_ref, 1e-11)


def test_concurrent_equals_sequential():
    from paper_2407_09621_gb300 import _lib
    probs = batch_problems(count=5, seed_base=3000, cells_choices=(8, 16), degrees=(2, 3))
    r_seq, _ = _lib.tp_batch_solve(probs, streams=1)
    r_con, _ = _lib.tp_batch_solve(probs, streams=5)
    for a, b in zip(r_seq, r_con):
        assert a["iterations"] == b["iterations"]
        assert abs(a["l2_error"] - b["l2_error"]) <= 1e-12 + 1e-9 * a["l2_error"]


def test_batch_over_caller_solvers_matches_exact_discrete_solutions():
    """tp_batch_solve_solvers: the caller's own (solver, x, b) entries of uneven sizes and degrees,
    solved concurrently, each against its exact discrete solution; a solver listed twice is
    rejected before any work."""
    from paper_2407_09621_gb300 import _lib
    from oracle.solve import rhs_sine
    specs = [(8, 2), (6, 3), (4, 5), (5, 1)]
    objs, xs, bs = [], [], []
    try:
        for nc, k in specs:
            mesh = _lib.tp_mesh_create(nc, nc, nc)
            op = _lib.tp_dg_laplace_create(mesh, k, _lib.TP_FP64)
            mg = _lib.tp_mg_create(op, precision=_lib.TP_FP32, coarse_cells=2)
            solver = _lib.tp_fgmres_create(op, mg, 30)
            objs.append((mesh, op, mg, solver))
            bs.append(torch.from_numpy(rhs_sine(k, nc, nc, nc)).cuda())
            xs.append(torch.zeros_like(bs[-1]))
        infos, sts, total = _lib.tp_batch_solve_solvers([o[3] for o in objs], [x.data_ptr() for x in xs],
                                                        [b.data_ptr() for b in bs], streams=3)
        assert total > 0 and sts == [0] * len(specs)
        for (nc, k), x, info in zip(specs, xs, infos):
            assert info["converged"] == 1
            u = FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))
            assert rel_l2(x.cpu().numpy(), u) < 1e-7
        with pytest.raises(_lib.TPError):
            _lib.tp_batch_solve_solvers([objs[0][3], objs[0][3]], [xs[0].data_ptr()] * 2, [bs[0].data_ptr()] * 2)
    finally:
        for mesh, op, mg, solver in objs:
            _lib.tp_solver_destroy(solver)
            _lib.tp_mg_destroy(mg)
            _lib.tp_op_destroy(op)
            _lib.tp_mesh_destroy(mesh)
