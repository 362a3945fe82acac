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


@pytest.mark.parametrize("autotune", [0, 1])
def test_small_uneven_batch_matches_oracle(autotune):
    from paper_2407_09621_gb300 import _lib
    probs = batch_problems(count=6, seed_base=2000, cells_choices=(4, 6, 8), degrees=(1, 2, 3, 4, 5, 6, 7))
    xs = []
    for p in probs:
        xs.append(torch.zeros(p["dofs"], dtype=torch.float64, device="cuda"))
        p["x_ptr"] = xs[-1].data_ptr()
    res, total = _lib.tp_batch_solve(probs, streams=4, autotune=autotune)
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
