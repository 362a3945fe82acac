"""GPU parity of tp_apply against the CPU oracle (element by element).

Small meshes: every entry against the assembled SIPG matrix (or its block
form, pinned to it). Full-size meshes: sampled cells computed one by one
from the element and face matrices, plus the rank-1 closed form of
Eq. (9), which holds at any size. Tolerances are relative l2 errors
(Sec. 5.2): 1e-12 FP64, 1e-5 FP32, 5e-3 FP16/BF16.
"""
import numpy as np
import pytest
import torch

from oracle.sipg import Mesh, assemble, BlockOperator, global_1d, kron_apply
from tp_synth import uniform_vector, sample_cells
from tests.gpu_util import TOL, DTYPES, rel_l2, to_device, to_host64

pytestmark = pytest.mark.gpu

torch_ok = torch.cuda.is_available()


def _gpu_apply(dims, k, prec, x64, kernel=0, penalty=0, lengths=(1.0, 1.0, 1.0)):
    from paper_2407_09621_gb300 import DGLaplace
    op = DGLaplace(*dims, k, prec, penalty=penalty, kernel=kernel, lengths=lengths)
    try:
        x = to_device(x64, prec)
        y = torch.empty_like(x)
        op.apply(y, x)
        torch.cuda.synchronize()
        return to_host64(y)
    finally:
        op.close()


def test_config0_fp64_8cubed_k3_full_matrix():
    # 8^3 cells, k = 3, x ~ U[-1,1] seed 0: every entry against the assembled matrix
    m = Mesh(8, 8, 8)
    A = assemble(m, 3)
    x = uniform_vector(A.shape[0], seed=0)
    y = _gpu_apply((8, 8, 8), 3, "fp64", x)
    ref = A @ x
    assert rel_l2(y, ref) < TOL["fp64"]
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("k", range(1, 8))
@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 2, 5), (5, 1, 2), (2, 7, 1)])
def test_fp64_all_degrees_ragged_meshes(k, dims):
    m = Mesh(*dims)
    bo = BlockOperator(m, k)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=k)
    y = _gpu_apply(dims, k, "fp64", x)
    ref = bo.apply(x)
    assert rel_l2(y, ref) < TOL["fp64"]
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("pen", [0, 1])
def test_fp64_paper_penalty_and_anisotropic_box(pen):
    dims, k, lengths = (4, 3, 2), 2, (0.7, 1.9, 0.45)
    m = Mesh(*dims, *lengths)
    A = assemble(m, k, "paper" if pen else "config")
    x = uniform_vector(A.shape[0], seed=3)
    y = _gpu_apply(dims, k, "fp64", x, penalty=pen, lengths=lengths)
    assert rel_l2(y, A @ x) < TOL["fp64"]


def _auto_differs(k, prec):
    """AUTO resolves to tcgen05 for FP16/BF16 vectors at k = 3 and to the CUDA-core kernel elsewhere."""
    return k == 3 and prec in ("fp16", "bf16")


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("kernel", [0, 1])
def test_low_precision_against_fp64_oracle(prec, k, kernel):
    if kernel == 1 and not _auto_differs(k, prec):
        pytest.skip("AUTO already is the CUDA-core kernel here")
    dims = (5, 3, 4)
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=10 + k)
    y = _gpu_apply(dims, k, prec, x, kernel=kernel)
    assert rel_l2(y, BlockOperator(m, k).apply(x)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("dims", [(17, 9, 13), (1, 1, 1), (2, 1, 7), (130, 2, 1)])
def test_cell_per_thread_kernel_k1(prec, dims):
    """At k = 1 the CUDA-core apply with FP32 arithmetic runs one thread per cell (128 cells per
    block): meshes over several blocks with a ragged last block, and one-cell and one-cell-thick
    meshes where most faces are boundary faces, against the oracle."""
    from paper_2407_09621_gb300 import DGLaplace
    m = Mesh(*dims)
    x64 = uniform_vector(m.ncells * 8, seed=91)
    op = DGLaplace(*dims, 1, prec, kernel=1)
    try:
        assert op.info["tile_cells"] == 128
        x = to_device(x64, prec)
        y = torch.empty_like(x)
        op.apply(y, x)
        torch.cuda.synchronize()
        assert rel_l2(y.double().cpu().numpy(), BlockOperator(m, 1).apply(x64)) < TOL[prec]
    finally:
        op.close()


@pytest.mark.parametrize("k", range(1, 8))
@pytest.mark.parametrize("dims", [(13, 9, 11), (1, 1, 1), (3, 1, 7)])
def test_double_word_fp64_apply_matches_oracle(k, dims):
    """FP64 vectors in double-word FP32 arithmetic (tp_op_opts.dword): within the FP64 tolerance
    of the oracle on meshes over several blocks and on one-cell and one-cell-thick meshes, and
    within 1e-13 of the FP64 kernel."""
    from paper_2407_09621_gb300 import DGLaplace
    m = Mesh(*dims)
    x64 = uniform_vector(m.ncells * (k + 1) ** 3, seed=95 + k)
    x = torch.from_numpy(x64).cuda()
    ys = []
    for dword in (0, 1):
        op = DGLaplace(*dims, k, "fp64", kernel=1, dword=dword)
        try:
            assert op.info["dword"] == dword and op.info["kernel"] == 1
            y = torch.empty_like(x)
            op.apply(y, x)
            torch.cuda.synchronize()
            ys.append(y.cpu().numpy())
        finally:
            op.close()
    assert rel_l2(ys[1], BlockOperator(m, k).apply(x64)) < TOL["fp64"]
    assert rel_l2(ys[1], ys[0]) < 1e-13


def test_double_word_host_apply_matches_device():
    """tp_apply_host on a double-word operator runs the same kernel over z-slab chunks: equal to
    tp_apply bit for bit."""
    from paper_2407_09621_gb300 import DGLaplace
    dims, k = (6, 5, 17), 3
    m = Mesh(*dims)
    x64 = uniform_vector(m.ncells * 64, seed=97)
    op = DGLaplace(*dims, k, "fp64", dword=1)
    try:
        xd = torch.from_numpy(x64).cuda()
        yd = torch.empty_like(xd)
        op.apply(yd, xd)
        xh = xd.cpu().pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        op.apply_host(yh, xh)
        torch.cuda.synchronize()
        assert torch.equal(yh, yd.cpu())
        assert rel_l2(yh.numpy(), BlockOperator(m, k).apply(x64)) < TOL["fp64"]
    finally:
        op.close()


@pytest.mark.parametrize("k,prec,family,path", [(3, "fp16", 2, 2), (3, "bf16", 2, 2), (3, "fp64", 1, 0),
                                                (3, "fp32", 1, 0), (2, "fp16", 1, 0), (7, "bf16", 1, 0),
                                                (7, "fp64", 1, 0), (12, "fp32", 1, 0)])
def test_auto_kernel_selection(k, prec, family, path):
    """TP_KERNEL_AUTO takes the family measured fastest for the precision and degree."""
    from paper_2407_09621_gb300 import DGLaplace
    op = DGLaplace(3, 2, 4, k, prec)
    try:
        assert op.info["kernel"] == family and op.info["tensor_path"] == path
        assert op.info["approximate"] == 0
    finally:
        op.close()


@pytest.mark.parametrize("tc_type,ec,approx", [(2, 1, 0), (2, 0, 1), (2, 2, 1), (2, 3, 1), (3, 1, 1), (3, 0, 1)])
def test_fp32_tensor_operators_flag_their_accuracy(tc_type, ec, approx):
    """FP32 vectors on the half-precision tensor path reach FP32 accuracy only with FP16 operands
    and both operands refined; every other combination reports itself as approximate."""
    from paper_2407_09621_gb300 import DGLaplace
    op = DGLaplace(3, 3, 3, 3, "fp32", kernel=TENSOR, ec=ec, tc_type=tc_type)
    try:
        assert op.info["approximate"] == approx
    finally:
        op.close()


def test_apply_is_deterministic_fp64():
    x = uniform_vector(6 * 5 * 4 * 64, seed=4)
    a = _gpu_apply((6, 5, 4), 3, "fp64", x)
    b = _gpu_apply((6, 5, 4), 3, "fp64", x)
    assert np.array_equal(a, b)


def test_host_buffer_entry_point_matches_device():
    from paper_2407_09621_gb300 import DGLaplace
    dims, k = (4, 4, 4), 3
    x = uniform_vector(64 * 64, seed=7)
    op = DGLaplace(*dims, k, "fp64")
    try:
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        op.apply_host(yh, xh)
        yd = torch.empty(op.ndofs, dtype=torch.float64, device="cuda")
        op.apply(yd, xh.cuda())
        torch.cuda.synchronize()
        assert np.array_equal(yh.numpy(), yd.cpu().numpy())
    finally:
        op.close()


def test_invalid_device_arguments_rejected():
    from paper_2407_09621_gb300 import DGLaplace, _lib
    op = DGLaplace(2, 2, 2, 2, "fp64")
    try:
        x = torch.zeros(op.ndofs + 8, dtype=torch.float64, device="cuda")
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_apply(op.op, x.data_ptr() + 8, x.data_ptr(), 0)  # overlapping
        assert e.value.status == _lib.TP_ERR_INVALID_ARG
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_apply(op.op, x.data_ptr() + 8, x.data_ptr() + 4, 0)  # unaligned
        assert e.value.status == _lib.TP_ERR_INVALID_ARG
    finally:
        op.close()


def _rank1_vectors(k, nc, seed):
    """x = c (x) b (x) a and, by Eq. (9) with the global 1D factors,
    A x = L c (x) M b (x) M a + M c (x) L b (x) M a + M c (x) M b (x) L a, cell-major order.
    Exact for any 1D vectors, so it checks every entry at any mesh size."""
    M, L = global_1d(k, nc)
    rng = np.random.default_rng(seed)
    n = k + 1
    nodes = np.concatenate([(c + np.linspace(0, 1, n)) / nc for c in range(nc)])
    a, b = rng.uniform(-1, 1, (2, nc * n))
    c = np.sin(np.pi * nodes)  # one smooth factor
    r = lambda v: v.reshape(nc, n)
    t = lambda vz, vy, vx: np.einsum("zl,yj,xi->zyxlji", r(vz), r(vy), r(vx), optimize=True).reshape(-1)
    x = t(c, b, a)
    y = t(L @ c, M @ b, M @ a) + t(M @ c, L @ b, M @ a) + t(M @ c, M @ b, L @ a)
    return x, y


@pytest.mark.parametrize("k,nc", [(3, 128), (7, 64)])
def test_config1_full_size_fp64_sampled_and_rank1(k, nc):
    # 134,217,728 DoFs: sampled cells against the oracle's element/face matrices
    dims = (nc, nc, nc)
    m = Mesh(*dims)
    ndofs = m.ncells * (k + 1) ** 3
    x = uniform_vector(ndofs, seed=0)
    y = _gpu_apply(dims, k, "fp64", x)
    cells = sample_cells(m.ncells, 1024 if k == 7 else 4096, seed=1, nx=nc, ny=nc, nz=nc)
    ref = BlockOperator(m, k).rows(x, cells)
    got = y.reshape(m.ncells, -1)[cells]
    assert rel_l2(got, ref) < TOL["fp64"]
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    del x, y
    # rank-1 closed form of Eq. (9) on every entry
    xs, ys = _rank1_vectors(k, nc, seed=17)
    y2 = _gpu_apply(dims, k, "fp64", xs)
    assert rel_l2(y2, ys) < TOL["fp64"]


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("k,nc", [(2, 107), (3, 80), (4, 64), (5, 54), (7, 40)])
@pytest.mark.parametrize("kernel", [0, 1])
def test_config2_precision_sweep_sampled(prec, k, nc, kernel):
    if kernel == 1 and not _auto_differs(k, prec):
        pytest.skip("AUTO already is the CUDA-core kernel here")
    dims = (nc, nc, nc)
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=0)
    y = _gpu_apply(dims, k, prec, x, kernel=kernel)
    cells = sample_cells(m.ncells, 512, seed=2, nx=nc, ny=nc, nz=nc)
    ref = BlockOperator(m, k).rows(x, cells)
    assert rel_l2(y.reshape(m.ncells, -1)[cells], ref) < TOL[prec]


# ---------------------------------------------------------------- FP64 tensor-core (DMMA) kernel
TENSOR = 2


@pytest.mark.parametrize("k", [3, 7])
@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 3, 4), (9, 2, 1), (2, 1, 11)])
def test_fp64_dmma_ragged_meshes(k, dims):
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=50 + k)
    y = _gpu_apply(dims, k, "fp64", x, kernel=TENSOR)
    assert rel_l2(y, BlockOperator(m, k).apply(x)) < TOL["fp64"]


def test_fp64_dmma_full_matrix_paper_penalty_anisotropic():
    dims, k = (4, 3, 5), 3
    m = Mesh(*dims, 1.0, 0.5, 2.0)
    A = assemble(m, k, "paper")
    x = uniform_vector(A.shape[0], seed=8)
    y = _gpu_apply(dims, k, "fp64", x, kernel=TENSOR, penalty=1, lengths=(1.0, 0.5, 2.0))
    assert rel_l2(y, A @ x) < TOL["fp64"]


@pytest.mark.parametrize("k,nc", [(3, 128), (7, 64)])
def test_config1_full_size_fp64_dmma(k, nc):
    """The 134M-DoF configurations on the DMMA kernel: rank-1 closed form of Eq. (9) on every
    entry, and agreement with the CUDA-core kernel on a random vector."""
    from paper_2407_09621_gb300 import DGLaplace
    dims = (nc, nc, nc)
    op = DGLaplace(*dims, k, "fp64", kernel=TENSOR)
    try:
        assert op.info["tensor_path"] == 3
    finally:
        op.close()
    xs, ys = _rank1_vectors(k, nc, seed=17)
    y2 = _gpu_apply(dims, k, "fp64", xs, kernel=TENSOR)
    assert rel_l2(y2, ys) < TOL["fp64"]
    del xs, ys, y2
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * (k + 1) ** 3, seed=0)
    cells = sample_cells(m.ncells, 1024, seed=3, nx=nc, ny=nc, nz=nc)
    y = _gpu_apply(dims, k, "fp64", x, kernel=TENSOR)
    ref = BlockOperator(m, k).rows(x, cells)
    assert rel_l2(y.reshape(m.ncells, -1)[cells], ref) < TOL["fp64"]


@pytest.mark.parametrize("k", [1, 2, 4, 5, 6])
def test_fp64_dmma_other_degrees_rejected(k):
    from paper_2407_09621_gb300 import DGLaplace, TPError
    with pytest.raises(TPError):
        DGLaplace(2, 2, 2, k, "fp64", kernel=TENSOR)


# ---------------------------------------------------------------- tile-shape autotuner
CC = 1


@pytest.mark.parametrize("k,prec,kernel", [(3, "fp64", CC), (7, "fp64", CC), (2, "fp32", CC), (3, "fp16", CC),
                                           (5, "bf16", CC), (3, "fp64", TENSOR), (7, "fp64", TENSOR)])
def test_autotuned_apply_identical_to_default(k, prec, kernel):
    """The autotuner only changes cells per thread block; every cell's arithmetic is unchanged,
    so the tuned operator's output equals the default one bit for bit, and matches the oracle."""
    from paper_2407_09621_gb300 import DGLaplace
    dims = (13, 9, 11)
    m = Mesh(*dims)
    x64 = uniform_vector(m.ncells * (k + 1) ** 3, seed=60 + k)
    outs, tiles = [], []
    for tune in (0, 1):
        op = DGLaplace(*dims, k, prec, kernel=kernel, autotune=tune)
        try:
            tiles.append(op.info["tile_cells"])
            x = to_device(x64, prec)
            y = torch.empty_like(x)
            op.apply(y, x)
            torch.cuda.synchronize()
            outs.append(y.cpu())
        finally:
            op.close()
    base = (128 // (k + 1) ** 2) or 1
    if kernel == TENSOR:
        base = 4 if k == 7 else 8
    elif m.ncells < 2 * torch.cuda.get_device_properties(0).multi_processor_count * base:
        base = max(base // 2, 1)  # small meshes default to the half-size CUDA-core tile
    assert tiles[0] == base and tiles[1] in (max(base // 2, 1), base, 2 * base, 4 * base)
    assert torch.equal(outs[0], outs[1])
    assert rel_l2(outs[1].double().numpy(), BlockOperator(m, k).apply(x64)) < TOL[prec]


@pytest.mark.parametrize("k,prec,kernel,dims,pinned", [
    (3, "fp64", 0, (6, 5, 8), True), (3, "fp64", 0, (7, 3, 11), False), (2, "fp32", 0, (5, 6, 19), True),
    (1, "fp32", 0, (9, 5, 17), True), (1, "bf16", 0, (4, 7, 10), False),
    (7, "fp64", TENSOR, (3, 4, 9), True), (3, "fp16", TENSOR, (9, 4, 10), True), (3, "bf16", 0, (4, 4, 8), True)])
def test_pipelined_host_apply_matches_device(k, prec, kernel, dims, pinned):
    """tp_apply_host cuts meshes with at least eight z-layers into z-slab chunks whose copies and
    applies overlap (CUDA-core and DMMA kernels); the result must equal tp_apply bit for bit,
    with pinned or pageable host memory, for chunk sizes that do not divide nz."""
    from paper_2407_09621_gb300 import DGLaplace
    m = Mesh(*dims)
    x64 = uniform_vector(m.ncells * (k + 1) ** 3, seed=71)
    op = DGLaplace(*dims, k, prec, kernel=kernel)
    try:
        xd = to_device(x64, prec)
        xh = xd.cpu()
        yh = torch.empty_like(xh)
        if pinned:
            xh, yh = xh.pin_memory(), yh.pin_memory()
        for _ in range(2):  # second call reuses the staging buffers and the pipeline
            yh.fill_(0)
            op.apply_host(yh, xh)
        yd = torch.empty_like(xd)
        op.apply(yd, xd)
        torch.cuda.synchronize()
        assert torch.equal(yh, yd.cpu())
        assert rel_l2(yh.double().numpy(), BlockOperator(m, k).apply(x64)) < TOL[prec]
    finally:
        op.close()


# ---------------------------------------------------------------- degrees 8..15 (CUDA-core, FP64 and FP32)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", range(8, 16))
def test_high_degrees_ragged_meshes(k, prec):
    """n = 9..16 nodes per direction (the arbitrary-size range of the paper's appendix): every
    entry against the Kronecker-sum form of Eq. (9), on meshes with one, two and three cells per
    direction (interior faces, boundary faces and both on one cell)."""
    for dims in [(3, 2, 2), (1, 3, 1)]:
        x = uniform_vector(int(np.prod(dims)) * (k + 1) ** 3, seed=80 + k)
        y = _gpu_apply(dims, k, prec, x)
        ref = kron_apply(x, k, dims)
        assert rel_l2(y, ref) < TOL[prec]
        if prec == "fp64":
            assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()


def test_high_degree_block_operator_k8():
    # the element/face block rows at k = 8, the oracle path that is independent of the 1D factors
    dims = (2, 3, 2)
    m = Mesh(*dims)
    x = uniform_vector(m.ncells * 9 ** 3, seed=88)
    assert rel_l2(_gpu_apply(dims, 8, "fp64", x), BlockOperator(m, 8).apply(x)) < TOL["fp64"]


@pytest.mark.parametrize("pen", [0, 1])
def test_high_degree_paper_penalty_anisotropic_box(pen):
    dims, k, lengths = (2, 3, 2), 13, (0.7, 1.9, 0.45)
    x = uniform_vector(int(np.prod(dims)) * (k + 1) ** 3, seed=90 + pen)
    y = _gpu_apply(dims, k, "fp64", x, penalty=pen, lengths=lengths)
    assert rel_l2(y, kron_apply(x, k, dims, lengths, "paper" if pen else "config")) < TOL["fp64"]


@pytest.mark.parametrize("k,nc", [(8, 32), (11, 24), (15, 20)])
def test_high_degree_full_size_rank1(k, nc):
    # 23.9M - 32.8M DoFs: the rank-1 closed form of Eq. (9) on every entry
    xs, ys = _rank1_vectors(k, nc, seed=19)
    y = _gpu_apply((nc, nc, nc), k, "fp64", xs)
    assert rel_l2(y, ys) < TOL["fp64"]
    y32 = _gpu_apply((nc, nc, nc), k, "fp32", xs)
    assert rel_l2(y32, ys) < TOL["fp32"]


@pytest.mark.parametrize("k,prec", [(9, "fp64"), (14, "fp32")])
def test_high_degree_pipelined_host_apply(k, prec):
    # tp_apply_host's z-slab pipeline with n > 8 equals tp_apply bit for bit
    from paper_2407_09621_gb300 import DGLaplace
    dims = (2, 2, 9)
    x64 = uniform_vector(36 * (k + 1) ** 3, seed=95)
    op = DGLaplace(*dims, k, prec)
    try:
        assert op.info["tile_cells"] == 1
        xd = to_device(x64, prec)
        xh = xd.cpu().pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        op.apply_host(yh, xh)
        yd = torch.empty_like(xd)
        op.apply(yd, xd)
        torch.cuda.synchronize()
        assert torch.equal(yh, yd.cpu())
        assert rel_l2(yh.double().numpy(), kron_apply(x64, k, dims)) < TOL[prec]
    finally:
        op.close()


def test_high_degree_autotune_keeps_single_tile_and_rejects_multigrid():
    from paper_2407_09621_gb300 import DGLaplace, _lib
    op = DGLaplace(4, 4, 4, 10, "fp64", autotune=1)
    try:
        assert op.info["tile_cells"] == 1 and op.info["k"] == 10
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_mg_create(op.op)
        assert e.value.status == _lib.TP_ERR_UNSUPPORTED
        u = torch.zeros(op.ndofs, dtype=torch.float64, device="cuda")
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_l2_error_sines(op.op, u.data_ptr())
        assert e.value.status == _lib.TP_ERR_UNSUPPORTED
    finally:
        op.close()


@pytest.mark.parametrize("k", range(1, 16))
def test_flops_per_dof_reports_the_contraction_form(k):
    """n >= 5 takes the even-odd form of the centrosymmetric 1D matrices: a line costs n^2/2 FMAs
    and 2n adds (even n) or (n^2 + 1)/2 FMAs and 2(n - 1) adds (odd n) instead of n^2 FMAs."""
    from paper_2407_09621_gb300 import DGLaplace
    n = k + 1
    op = DGLaplace(2, 2, 2, k, "fp64")
    try:
        if n >= 5:
            line = n * n + 2 * n if n % 2 == 0 else n * n + 1 + 2 * (n - 1)
        else:
            line = 2 * n * n
        assert op.info["flops_per_dof"] == pytest.approx(6 * line / n + 38)
    finally:
        op.close()
