"""GPU parity of the multigrid steps, the V-cycle and the FGMRES solve against
the CPU oracle (oracle/mg.py, oracle/solve.py).

Each step of Algorithm 2 is compared element by element with the oracle on
the same seeded inputs and the same explicit smoother bound lmax (an input
of both sides); the solve is compared with the exact discrete solution by
fast diagonalization and by the L2 error rule (within 1% of the FP64 solve's
discretization error, or at the round-off floor when that error is below
1e-10)."""
import numpy as np
import pytest
import torch

from oracle.mg import VCycle, prolongation, chebyshev, jacobi_diagonal, fgmres
from oracle.sipg import Mesh, BlockOperator
from oracle.solve import FastDiag, rhs_sine, l2_error, sine_exact
from tp_synth import uniform_vector
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu

DT = {"fp64": torch.float64, "fp32": torch.float32, "fp16": torch.float16, "bf16": torch.bfloat16}
TOLS = {"fp64": 1e-12, "fp32": 1e-5}
PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}


class GpuMG:
    def __init__(self, nc, k, prec, lmax=0.0, coarse_cells=1, degree=3, smoother=0, dims=None, kernel=1):
        from paper_2407_09621_gb300 import _lib
        self.lib = _lib
        self.mesh = _lib.tp_mesh_create(*(dims or (nc, nc, nc)))
        self.op = _lib.tp_dg_laplace_create(self.mesh, k, _lib.TP_FP64)
        self.mg = _lib.tp_mg_create(self.op, degree=degree, lmax=lmax, coarse_cells=coarse_cells,
                                    precision=PREC[prec], smoother=smoother, kernel=kernel)
        self.info = _lib.tp_mg_get_info(self.mg)
        self.dtype = DT[prec]

    def vec(self, x64):
        return torch.from_numpy(np.ascontiguousarray(x64)).to("cuda", self.dtype)

    def close(self):
        self.lib.tp_mg_destroy(self.mg)
        self.lib.tp_op_destroy(self.op)
        self.lib.tp_mesh_destroy(self.mesh)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 7])
def test_transfer_matches_oracle(prec, k):
    g = GpuMG(4, k, prec, lmax=3.0, coarse_cells=1)
    try:
        L = g.info["levels"]
        for level in (L - 1, L - 2):
            ncc = g.info["cells"][level - 1][0]
            P = prolongation(k, ncc, ncc, ncc)
            fine = uniform_vector(P.shape[0], seed=level)
            coarse = uniform_vector(P.shape[1], seed=level + 50)
            dc = torch.empty(P.shape[1], dtype=g.dtype, device="cuda")
            g.lib.tp_mg_restrict(g.mg, level, dc.data_ptr(), g.vec(fine).data_ptr())
            df = g.vec(fine)
            g.lib.tp_mg_prolongate_add(g.mg, level, df.data_ptr(), g.vec(coarse).data_ptr())
            torch.cuda.synchronize()
            assert rel_l2(dc.double().cpu().numpy(), P.T @ fine) < TOLS[prec]
            assert rel_l2(df.double().cpu().numpy(), fine + P @ coarse) < TOLS[prec]
    finally:
        g.close()


@pytest.mark.parametrize("k,nc", [(1, 2), (3, 2), (7, 1), (2, 3)])
def test_coarse_solve_matches_fast_diagonalization(k, nc):
    g = GpuMG(nc, k, "fp64", lmax=3.0, coarse_cells=8)
    try:
        assert g.info["levels"] == 1
        b = uniform_vector(nc ** 3 * (k + 1) ** 3, seed=9)
        x = torch.empty(len(b), dtype=torch.float64, device="cuda")
        g.lib.tp_mg_coarse_solve(g.mg, x.data_ptr(), g.vec(b).data_ptr())
        torch.cuda.synchronize()
        assert rel_l2(x.cpu().numpy(), FastDiag(k, nc, nc, nc).solve(b)) < 1e-11
    finally:
        g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_smoother_matches_oracle(prec, k):
    nc, lmax = 4, 2.8
    g = GpuMG(nc, k, prec, lmax=lmax, coarse_cells=2)
    try:
        fl = g.info["levels"] - 1
        n = g.info["ndofs"][fl]
        b, x0 = uniform_vector(n, seed=1), uniform_vector(n, seed=2)
        x = g.vec(x0)
        g.lib.tp_mg_smooth(g.mg, fl, x.data_ptr(), g.vec(b).data_ptr())
        torch.cuda.synchronize()
        A = BlockOperator(Mesh(nc, nc, nc), k)
        ref = chebyshev(A.apply, 1.0 / jacobi_diagonal(k, nc, nc, nc), b, x0, lmax, 3, 15.0)
        assert rel_l2(x.double().cpu().numpy(), ref) < (1e-12 if prec == "fp64" else 2e-5)
    finally:
        g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,nc,cnc", [(3, 8, 1), (2, 8, 2), (7, 4, 1), (1, 16, 4)])
def test_vcycle_matches_oracle(prec, k, nc, cnc):
    lmax = 2.9 if k > 1 else 4.9
    g = GpuMG(nc, k, prec, lmax=lmax, coarse_cells=cnc)
    try:
        n = g.info["ndofs"][-1]
        b, x0 = uniform_vector(n, seed=3), uniform_vector(n, seed=4)
        x = g.vec(x0)
        g.lib.tp_vcycle(g.mg, x.data_ptr(), g.vec(b).data_ptr())
        torch.cuda.synchronize()
        mg = VCycle(k, nc, coarse_nc=cnc)
        mg.lmax = [None] + [lmax] * (len(mg.levels) - 1)
        ref = mg.vcycle(len(mg.levels) - 1, b, x0)
        assert len(mg.levels) == g.info["levels"]
        assert rel_l2(x.double().cpu().numpy(), ref) < (1e-11 if prec == "fp64" else 5e-5)
    finally:
        g.close()


@pytest.mark.parametrize("k", [1, 3, 7])
def test_lmax_estimate_bounds_the_spectrum(k):
    import scipy.sparse.linalg as spla
    nc = 4
    g = GpuMG(nc, k, "fp64", lmax=0.0, coarse_cells=2)
    try:
        est = g.info["lmax"][-1] / 1.1
        A = BlockOperator(Mesh(nc, nc, nc), k)
        dinv = 1.0 / jacobi_diagonal(k, nc, nc, nc)
        n = len(dinv)
        op = spla.LinearOperator((n, n), matvec=lambda v: np.sqrt(dinv) * A.apply(np.sqrt(dinv) * v))
        exact = spla.eigsh(op, k=1, which="LA", tol=1e-8)[0][0]
        assert 0.9 * exact <= est <= exact * (1 + 1e-6)
        assert g.info["lmax"][-1] >= 0.99 * exact
    finally:
        g.close()


def _solve(nc, k, mg_prec, rtol=1e-10, maxit=200, lmax=0.0, coarse_cells=4, kernel=1, smoother=0, dword=0):
    from paper_2407_09621_gb300 import _lib
    mesh = _lib.tp_mesh_create(nc, nc, nc)
    op = _lib.tp_dg_laplace_create(mesh, k, _lib.TP_FP64, dword=dword)
    mg = (_lib.tp_mg_create(op, lmax=lmax, coarse_cells=coarse_cells, precision=PREC[mg_prec], kernel=kernel,
                            smoother=smoother)
          if mg_prec else None)
    solver = _lib.tp_fgmres_create(op, mg, 30)
    try:
        b = torch.from_numpy(rhs_sine(k, nc, nc, nc)).cuda()
        x = torch.zeros_like(b)
        st, info = _lib.tp_fgmres_solve(solver, x.data_ptr(), b.data_ptr(), rtol, maxit)
        torch.cuda.synchronize()
        return x.cpu().numpy(), info
    finally:
        _lib.tp_solver_destroy(solver)
        if mg:
            _lib.tp_mg_destroy(mg)
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)


@pytest.mark.parametrize("mg_prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,nc", [(3, 16), (2, 16), (7, 8)])
def test_fgmres_solution_matches_exact_discrete_solution(mg_prec, k, nc):
    x, info = _solve(nc, k, mg_prec, lmax=2.9 if k > 1 else 4.9, coarse_cells=2)
    assert info["converged"] == 1
    assert info["true_rel_residual"] < 2e-10
    u = FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))
    assert rel_l2(x, u) < 1e-8
    # same preconditioned iteration count as the oracle's FGMRES within two steps
    mg = VCycle(k, nc, coarse_nc=2)
    mg.lmax = [None] + [2.9 if k > 1 else 4.9] * (len(mg.levels) - 1)
    A = BlockOperator(Mesh(nc, nc, nc), k)
    _, its, _ = fgmres(A.apply, mg, rhs_sine(k, nc, nc, nc), rtol=1e-10)
    assert abs(info["iterations"] - its) <= 2


@pytest.mark.parametrize("k,nc,smoother", [(3, 16, 0), (2, 16, 1), (7, 8, 1)])
def test_fgmres_double_word_arnoldi_products(k, nc, smoother):
    """With a double-word operator (tp_op_opts.dword) the Arnoldi products run in double-word FP32
    arithmetic and the residuals in FP64: the solve takes the FP64 operator's iteration count
    (within one), its true residual meets the tolerance and it reaches the exact discrete solution."""
    lmax = 2.9 if k > 1 else 4.9
    x_n, info_n = _solve(nc, k, "fp32", lmax=lmax, coarse_cells=2, smoother=smoother)
    x_d, info_d = _solve(nc, k, "fp32", lmax=lmax, coarse_cells=2, smoother=smoother, dword=1)
    assert info_d["converged"] == 1 and info_d["true_rel_residual"] < 2e-10
    assert abs(info_d["iterations"] - info_n["iterations"]) <= 1
    u = FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))
    assert rel_l2(x_d, u) < 1e-8 and rel_l2(x_d, x_n) < 1e-8


@pytest.mark.parametrize("kernel", [1, 2])
def test_fgmres_nonzero_initial_guess(kernel):
    """x0 near the solution: the initial residual is b - A x0 (the zero test of x0 must see it),
    on the CUDA-core FP64 operator (residual fused into the apply) and on the DMMA operator (apply,
    then the difference)."""
    from paper_2407_09621_gb300 import _lib
    k, nc = 3, 16
    mesh = _lib.tp_mesh_create(nc, nc, nc)
    op = _lib.tp_dg_laplace_create(mesh, k, _lib.TP_FP64, kernel=kernel)
    mg = _lib.tp_mg_create(op, coarse_cells=2, precision=PREC["fp32"])
    solver = _lib.tp_fgmres_create(op, mg, 30)
    try:
        f = rhs_sine(k, nc, nc, nc)
        u = FastDiag(k, nc, nc, nc).solve(f)
        b = torch.from_numpy(f).cuda()
        x = torch.from_numpy(u + 1e-3 * uniform_vector(len(u), seed=31)).cuda()
        st, info = _lib.tp_fgmres_solve(solver, x.data_ptr(), b.data_ptr(), 1e-8, 100)
        torch.cuda.synchronize()
        assert info["converged"] == 1 and info["iterations"] >= 1
        assert rel_l2(x.cpu().numpy(), u) < 1e-9
        x0 = torch.zeros_like(b)  # and from zero, the same solution
        st, info0 = _lib.tp_fgmres_solve(solver, x0.data_ptr(), b.data_ptr(), 1e-10, 100)
        torch.cuda.synchronize()
        assert info0["converged"] == 1 and rel_l2(x0.cpu().numpy(), u) < 1e-8
    finally:
        _lib.tp_solver_destroy(solver)
        _lib.tp_mg_destroy(mg)
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)


def test_fgmres_without_preconditioner_reports_not_converged():
    from paper_2407_09621_gb300 import _lib
    mesh = _lib.tp_mesh_create(4, 4, 4)
    op = _lib.tp_dg_laplace_create(mesh, 3, _lib.TP_FP64)
    solver = _lib.tp_fgmres_create(op, None, 10)
    try:
        b = torch.from_numpy(rhs_sine(3, 4, 4, 4)).cuda()
        x = torch.zeros_like(b)
        st, info = _lib.tp_fgmres_solve(solver, x.data_ptr(), b.data_ptr(), 1e-12, 5, raise_on_error=False)
        assert st == _lib.TP_ERR_NOT_CONVERGED and info["iterations"] == 5 and info["converged"] == 0
        assert len(info["history"]) == 6 and info["history"][-1] < 1.0
    finally:
        _lib.tp_solver_destroy(solver)
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)


def _l2_rule(e_mixed, e_fp64):
    if e_fp64 > 1e-10:
        return abs(e_mixed - e_fp64) <= 0.01 * e_fp64
    return e_mixed <= max(1.01 * e_fp64, 1e-11)


@pytest.mark.parametrize("k,nc", [(3, 64), (7, 32)])
def test_config3_mixed_solve_discretization_error(k, nc):
    # Poisson problem of Sec. 7.2 at full size: FP32 V-cycle inside FP64 FGMRES;
    # L2 error against the exact solution matches that of the exact discrete solution
    x, info = _solve(nc, k, "fp32")
    assert info["converged"] == 1
    u = FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))
    e_mixed = l2_error(x, k, nc, nc, nc, sine_exact)
    e_exact = l2_error(u, k, nc, nc, nc, sine_exact)
    assert _l2_rule(e_mixed, e_exact), (e_mixed, e_exact)


@pytest.mark.parametrize("k,nc", [(1, 3), (3, 4), (7, 2)])
def test_rhs_and_l2_error_match_oracle(k, nc):
    from oracle.solve import rhs_modes
    from paper_2407_09621_gb300 import _lib
    modes = [(0.7, 1, 2, 3), (-0.4, 3, 1, 1)]
    mesh = _lib.tp_mesh_create(nc, nc, nc)
    op = _lib.tp_dg_laplace_create(mesh, k, _lib.TP_FP64)
    try:
        n = _lib.tp_op_get_info(op)["ndofs"]
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        _lib.tp_rhs_sines(op, b.data_ptr(), modes)
        ref = rhs_modes(k, nc, nc, nc, modes)
        assert rel_l2(b.cpu().numpy(), ref) < 1e-13
        u = FastDiag(k, nc, nc, nc).solve(ref)
        exact = lambda X, Y, Z: sum(a * np.sin(p * np.pi * X) * np.sin(q * np.pi * Y) * np.sin(r * np.pi * Z)
                                    for a, p, q, r in modes)
        e_gpu = _lib.tp_l2_error_sines(op, torch.from_numpy(u).cuda().data_ptr(), modes)
        e_ref = l2_error(u, k, nc, nc, nc, exact)
        assert abs(e_gpu - e_ref) <= 1e-10 * e_ref
    finally:
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)


# ---------------------------------------------------------------- FP16 / BF16 storage V-cycles
@pytest.mark.parametrize("prec,tol", [("fp16", 1e-2), ("bf16", 5e-2)])
@pytest.mark.parametrize("k,nc,cnc", [(3, 8, 1), (2, 8, 2), (7, 4, 1)])
def test_half_storage_vcycle_matches_oracle(prec, tol, k, nc, cnc):
    """The V-cycle with FP16/BF16 vectors (FP32 arithmetic) against the FP64 oracle V-cycle:
    same algorithm, storage rounding only (2^-11 / 2^-8 per stored value)."""
    lmax = 2.9
    g = GpuMG(nc, k, prec, lmax=lmax, coarse_cells=cnc)
    try:
        assert g.info["precision"] == PREC[prec]
        n = g.info["ndofs"][-1]
        b, x0 = uniform_vector(n, seed=3), uniform_vector(n, seed=4)
        x = g.vec(x0)
        g.lib.tp_vcycle(g.mg, x.data_ptr(), g.vec(b).data_ptr())
        torch.cuda.synchronize()
        mg = VCycle(k, nc, coarse_nc=cnc)
        mg.lmax = [None] + [lmax] * (len(mg.levels) - 1)
        ref = mg.vcycle(len(mg.levels) - 1, b, x0)
        assert rel_l2(x.double().cpu().numpy(), ref) < tol
    finally:
        g.close()


@pytest.mark.parametrize("mg_prec", ["fp16", "bf16"])
@pytest.mark.parametrize("k,nc,kernel", [(3, 32, 1), (3, 32, 2), (2, 16, 2), (7, 16, 1)])
def test_half_vcycle_solve_meets_l2_rule(mg_prec, k, nc, kernel):
    """FP64 FGMRES preconditioned by an FP16/BF16-storage V-cycle (CUDA-core applies, or the
    tensor-core applies: tcgen05 at k = 3, mma.sync at k = 2) reaches the FP64 discretization
    error of Sec. 7.2."""
    x, info = _solve(nc, k, mg_prec, kernel=kernel, maxit=300)
    assert info["converged"] == 1
    u = FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))
    e_mixed = l2_error(x, k, nc, nc, nc, sine_exact)
    e_exact = l2_error(u, k, nc, nc, nc, sine_exact)
    assert _l2_rule(e_mixed, e_exact), (e_mixed, e_exact)


@pytest.mark.parametrize("k,nc", [(3, 16), (7, 8)])
def test_fgmres_basis_stays_orthonormal(k, nc):
    """Selective re-orthogonalization keeps the FGMRES basis orthonormal: after a solve the
    relative residual recomputed in FP64 matches the Arnoldi estimate (a lost orthogonality
    would show as a gap between the two), and the iteration count matches the oracle's
    modified Gram-Schmidt FGMRES within two."""
    x, info = _solve(nc, k, "fp32", lmax=2.9, coarse_cells=2)
    assert info["converged"] == 1
    assert info["true_rel_residual"] < 10 * max(info["rel_residual"], 1e-12)
    assert 0 <= info["reorthogonalizations"] <= info["iterations"]
    mg = VCycle(k, nc, coarse_nc=2)
    mg.lmax = [None] + [2.9] * (len(mg.levels) - 1)
    A = BlockOperator(Mesh(nc, nc, nc), k)
    _, its, _ = fgmres(A.apply, mg, rhs_sine(k, nc, nc, nc), rtol=1e-10)
    assert abs(info["iterations"] - its) <= 2


# ---------------------------------------------------------------- vertex-patch Schwarz smoother
VP = 1


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,dims", [(1, (4, 4, 4)), (2, (4, 6, 2)), (3, (4, 2, 4)), (2, (6, 4, 4)), (3, (4, 6, 4)),
                                    (5, (4, 4, 4))])
def test_vertex_patch_smoother_matches_oracle(prec, k, dims):
    """One sweep (colours ascending) on the finest level against the oracle's dense patch solves. With
    at least four cells in every direction some patches are interior ones (the even/odd bases)."""
    from oracle.schwarz import VertexPatchSmoother
    from oracle.sipg import assemble
    g = GpuMG(None, k, prec, coarse_cells=1, smoother=VP, dims=dims)
    try:
        fl = g.info["levels"] - 1
        n = g.info["ndofs"][fl]
        b, x0 = uniform_vector(n, seed=21), uniform_vector(n, seed=22)
        x = g.vec(x0)
        g.lib.tp_mg_smooth(g.mg, fl, x.data_ptr(), g.vec(b).data_ptr())
        torch.cuda.synchronize()
        ref = VertexPatchSmoother(assemble(Mesh(*dims), k), k, dims).smooth(x0, b)
        assert rel_l2(x.double().cpu().numpy(), ref) < (1e-12 if prec == "fp64" else 5e-5)
    finally:
        g.close()


@pytest.mark.parametrize("prec,k,kernel", [("fp64", 2, 1), ("fp32", 3, 1), ("fp32", 3, 2)])
def test_vertex_patch_smoother_on_anisotropic_box(prec, k, kernel):
    """Cells of different widths per direction (each direction's patch eigenbases from its own h and
    penalty), on CUDA-core or tensor-core (mma.sync, FP32 vectors) level operators."""
    from oracle.schwarz import VertexPatchSmoother
    from oracle.sipg import assemble
    from paper_2407_09621_gb300 import _lib
    dims, lengths = (4, 6, 2), (0.7, 1.3, 0.45)
    mesh = _lib.tp_mesh_create(*dims, *lengths)
    op = _lib.tp_dg_laplace_create(mesh, k, _lib.TP_FP64)
    # the tensor-core level operator with FP32 vectors runs with the error correction of Algorithm 1
    mg = _lib.tp_mg_create(op, coarse_cells=1, precision=PREC[prec], kernel=kernel, ec=int(kernel == 2), smoother=VP)
    try:
        info = _lib.tp_mg_get_info(mg)
        fl = info["levels"] - 1
        n = info["ndofs"][fl]
        b, x0 = uniform_vector(n, seed=27), uniform_vector(n, seed=28)
        x = torch.from_numpy(x0).to("cuda", DT[prec])
        _lib.tp_mg_smooth(mg, fl, x.data_ptr(), torch.from_numpy(b).to("cuda", DT[prec]).data_ptr())
        torch.cuda.synchronize()
        ref = VertexPatchSmoother(assemble(Mesh(*dims, *lengths), k), k, dims).smooth(x0, b)
        assert rel_l2(x.double().cpu().numpy(), ref) < (1e-12 if prec == "fp64" else 5e-5 if kernel == 1 else 2e-4)
    finally:
        _lib.tp_mg_destroy(mg)
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [1, 4, 5, 7])
def test_vertex_patch_single_patch_level_solves_exactly(prec, k):
    """2^3 cells: the only patch is the whole mesh, so one sweep from any x is A^{-1} b."""
    g = GpuMG(2, k, prec, coarse_cells=1, smoother=VP)
    try:
        fl = g.info["levels"] - 1
        n = g.info["ndofs"][fl]
        b, x0 = uniform_vector(n, seed=23), uniform_vector(n, seed=24)
        x = g.vec(x0)
        g.lib.tp_mg_smooth(g.mg, fl, x.data_ptr(), g.vec(b).data_ptr())
        torch.cuda.synchronize()
        ref = FastDiag(k, 2, 2, 2).solve(b)
        assert rel_l2(x.double().cpu().numpy(), ref) < (1e-11 if prec == "fp64" else 1e-4)
    finally:
        g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,nc,cnc", [(1, 8, 1), (2, 8, 2), (3, 4, 1)])
def test_vertex_patch_vcycle_matches_oracle(prec, k, nc, cnc):
    g = GpuMG(nc, k, prec, coarse_cells=cnc, smoother=VP)
    try:
        n = g.info["ndofs"][-1]
        b, x0 = uniform_vector(n, seed=25), uniform_vector(n, seed=26)
        x = g.vec(x0)
        g.lib.tp_vcycle(g.mg, x.data_ptr(), g.vec(b).data_ptr())
        torch.cuda.synchronize()
        mg = VCycle(k, nc, coarse_nc=cnc, smoother="vertex_patch")
        assert len(mg.levels) == g.info["levels"]
        ref = mg.vcycle(len(mg.levels) - 1, b, x0)
        assert rel_l2(x.double().cpu().numpy(), ref) < (1e-11 if prec == "fp64" else 5e-5)
    finally:
        g.close()


@pytest.mark.parametrize("mg_prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,nc", [(3, 16), (2, 16), (7, 8)])
def test_vertex_patch_solve_matches_exact_discrete_solution(mg_prec, k, nc):
    """FGMRES with the vertex-patch V-cycle: the exact discrete solution in at most six iterations
    (the Chebyshev-Jacobi V-cycle takes 12-15 on these problems)."""
    x, info = _solve(nc, k, mg_prec, coarse_cells=2, smoother=VP)
    assert info["converged"] == 1 and info["iterations"] <= 6
    assert info["true_rel_residual"] < 2e-10
    assert rel_l2(x, FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))) < 1e-8


@pytest.mark.parametrize("k,nc", [(3, 64), (7, 32)])
def test_vertex_patch_mixed_solve_discretization_error(k, nc):
    # FP32 vertex-patch V-cycle inside FP64 FGMRES at the Sec. 7.2 sizes: the L2 rule against the
    # exact discrete solution
    x, info = _solve(nc, k, "fp32", smoother=VP)
    assert info["converged"] == 1
    u = FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))
    e_mixed = l2_error(x, k, nc, nc, nc, sine_exact)
    e_exact = l2_error(u, k, nc, nc, nc, sine_exact)
    assert _l2_rule(e_mixed, e_exact), (e_mixed, e_exact)


@pytest.mark.parametrize("prec,tol", [("fp16", 1e-2), ("bf16", 5e-2)])
@pytest.mark.parametrize("k,nc,cnc,kernel", [(1, 8, 1, 1), (2, 8, 2, 1), (3, 4, 1, 1), (3, 8, 2, 2), (3, 4, 1, 2)])
def test_half_vertex_patch_vcycle_matches_oracle(prec, tol, k, nc, cnc, kernel):
    """The vertex-patch V-cycle with FP16/BF16 vectors (FP32 arithmetic; at k = 3 with kernel 2 the
    level residuals on tcgen05) against the FP64 oracle V-cycle: storage rounding only."""
    g = GpuMG(nc, k, prec, coarse_cells=cnc, smoother=VP, kernel=kernel)
    try:
        n = g.info["ndofs"][-1]
        b, x0 = uniform_vector(n, seed=27), uniform_vector(n, seed=28)
        x = g.vec(x0)
        g.lib.tp_vcycle(g.mg, x.data_ptr(), g.vec(b).data_ptr())
        torch.cuda.synchronize()
        mg = VCycle(k, nc, coarse_nc=cnc, smoother="vertex_patch")
        ref = mg.vcycle(len(mg.levels) - 1, b, x0)
        assert rel_l2(x.double().cpu().numpy(), ref) < tol
    finally:
        g.close()


@pytest.mark.parametrize("mg_prec", ["fp16", "bf16"])
@pytest.mark.parametrize("k,nc,kernel", [(3, 32, 2), (3, 32, 1), (7, 16, 1), (2, 16, 1)])
def test_half_vertex_patch_solve_meets_l2_rule(mg_prec, k, nc, kernel):
    """FP64 FGMRES preconditioned by an FP16/BF16-storage vertex-patch V-cycle reaches the FP64
    discretization error of Sec. 7.2 in a few iterations."""
    x, info = _solve(nc, k, mg_prec, kernel=kernel, maxit=100, smoother=VP)
    assert info["converged"] == 1 and info["iterations"] <= 12
    u = FastDiag(k, nc, nc, nc).solve(rhs_sine(k, nc, nc, nc))
    e_mixed = l2_error(x, k, nc, nc, nc, sine_exact)
    e_exact = l2_error(u, k, nc, nc, nc, sine_exact)
    assert _l2_rule(e_mixed, e_exact), (e_mixed, e_exact)


def test_mg_option_validation():
    from paper_2407_09621_gb300 import _lib
    mesh = _lib.tp_mesh_create(4, 4, 4)
    op = _lib.tp_dg_laplace_create(mesh, 3, _lib.TP_FP64)
    try:
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_mg_create(op, smoother=5)
        assert e.value.status == _lib.TP_ERR_INVALID_ARG
    finally:
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)


def _gpu_solve_l2(k, nc, prec, smoother):
    """FP64 FGMRES(30) to rtol 1e-10 with one V-cycle of `prec` and `smoother`; the L2 error of the
    solution against u = sin(pi x) sin(pi y) sin(pi z), evaluated on the GPU (tp_l2_error_sines,
    checked against the oracle's l2_error in test_rhs_and_l2_error_match_oracle)."""
    from paper_2407_09621_gb300 import _lib
    mesh = _lib.tp_mesh_create(nc, nc, nc)
    op = _lib.tp_dg_laplace_create(mesh, k, _lib.TP_FP64)
    mg = _lib.tp_mg_create(op, precision=PREC[prec], smoother=smoother)
    solver = _lib.tp_fgmres_create(op, mg, 30)
    try:
        n = _lib.tp_op_get_info(op)["ndofs"]
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        _lib.tp_rhs_sines(op, b.data_ptr())
        x = torch.zeros_like(b)
        st, info = _lib.tp_fgmres_solve(solver, x.data_ptr(), b.data_ptr(), 1e-10, 300)
        assert info["converged"] == 1
        return _lib.tp_l2_error_sines(op, x.data_ptr()), info
    finally:
        _lib.tp_solver_destroy(solver)
        _lib.tp_mg_destroy(mg)
        _lib.tp_op_destroy(op)
        _lib.tp_mesh_destroy(mesh)
        torch.cuda.empty_cache()


@pytest.mark.parametrize("k,nc", [(3, 128), (7, 64)])
def test_config3_full_size_mixed_solve_meets_l2_rule(k, nc):
    """The two 134M-DoF Poisson solves of Sec. 7.2's setting: the mixed solve (FP32 vertex-patch
    V-cycle) meets the L2 rule against the all-FP64 solve (FP64 Chebyshev V-cycle). The FP64 error is
    anchored to the oracle: at k = 3 within a factor 2 of the exact discrete solution's error on
    (nc/2)^3 cells divided by 2^(k+1) (the O(h^(k+1)) rate), at k = 7 at the FP64 round-off floor."""
    e64, info64 = _gpu_solve_l2(k, nc, "fp64", 0)
    e_mixed, info_mixed = _gpu_solve_l2(k, nc, "fp32", VP)
    if k == 3:
        h = nc // 2
        u = FastDiag(k, h, h, h).solve(rhs_sine(k, h, h, h))
        e_anchor = l2_error(u, k, h, h, h, sine_exact) / 2 ** (k + 1)
        assert 0.5 * e_anchor < e64 < 2.0 * e_anchor, (e64, e_anchor)
    else:
        assert e64 < 3e-11
    assert info_mixed["iterations"] <= 8
    assert _l2_rule(e_mixed, e64), (e_mixed, e64)
