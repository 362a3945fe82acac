"""tp_apply_host_noalloc: the host-buffer apply for callers that cannot call
cudaMalloc (their device memory is all taken by their own fixed pool, or they
must not meet the allocator mid-run). It stages through a static device array
instead of allocating, so its results must equal those of tp_apply_host,
which allocates its staging buffers. Two calls in a row check that nothing
left in the shared array from one call leaks into the next. This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from tp_synth import uniform_vector

pytestmark = pytest.mark.gpu


# kernel 0: the default (CUDA-core); 2: the tensor kernels (DMMA for FP64, tcgen05 with a TMA
# tensor map over the staged x for FP16 at k = 3)
@pytest.mark.parametrize("prec,dims,k,kernel", [("fp64", (4, 3, 5), 3, 0), ("fp32", (6, 6, 6), 2, 0),
                                                ("fp64", (8, 8, 8), 7, 0), ("fp64", (4, 4, 4), 3, 2),
                                                ("fp16", (4, 4, 4), 3, 2), ("bf16", (5, 3, 4), 3, 2)])
def test_noalloc_matches_allocating_host_apply(prec, dims, k, kernel):
    from paper_2407_09621_gb300 import DGLaplace, _lib
    op = DGLaplace(*dims, k, prec, kernel=kernel)
    try:
        assert op.ndofs * op.info["elem_bytes"] <= _lib.TP_NOALLOC_MAX_BYTES
        for seed in (11, 12):  # two calls in a row, different inputs
            x = torch.from_numpy(uniform_vector(op.ndofs, seed=seed)).to(op.dtype).pin_memory()
            y_ref = torch.empty_like(x).pin_memory()
            y_new = torch.full_like(x, float("nan")).pin_memory()
            _lib.tp_apply_host(op.op, y_ref.data_ptr(), x.data_ptr(), 0)
            _lib.tp_apply_host_noalloc(op.op, y_new.data_ptr(), x.data_ptr(), 0)
            op.check()  # no bounded device wait gave up
            a, b = y_new.double().numpy(), y_ref.double().numpy()
            # the same kernel on the same input: equal up to the storage rounding of the result
            tol = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 5e-3, "bf16": 5e-3}[prec]
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)
    finally:
        op.close()


def test_noalloc_rejects_vectors_beyond_the_limit():
    from paper_2407_09621_gb300 import DGLaplace, _lib
    op = DGLaplace(32, 32, 32, 3, "fp64")  # 2,097,152 doubles = 16 MiB > 8 MiB
    try:
        x = torch.zeros(op.ndofs, dtype=torch.float64)
        y = torch.zeros_like(x)
        st = _lib.lib.tp_apply_host_noalloc(op.op, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), None)
        assert st == _lib.TP_ERR_INVALID_ARG
        assert "limit" in _lib.tp_last_error()
    finally:
        op.close()
