"""Host-side checks of the C ABI: the library loads, exports every function the
header declares, and validates arguments (no GPU needed)."""
import ctypes

import pytest
import torch

from paper_2407_09621_gb300 import _lib


def test_header_functions_are_exported():
    names = _lib.header_functions()
    assert "tp_apply" in names and "tp_mesh_create" in names
    for name in names:
        assert hasattr(_lib.lib, name), f"{name} declared in include/tp.h but not exported"
        assert hasattr(_lib, name), f"{name} has no Python binding"


def test_bench_support_library_is_separate():
    """The measurement probes (include/tp_bench.h) live in libtp_bench.so, not in the method's library."""
    import os
    hdr = os.path.join(_lib.INCLUDE, "tp_bench.h")
    names = _lib.header_functions([hdr])
    assert "tp_bench_fma_peak" in names
    bench = ctypes.CDLL(os.path.join(_lib.HERE, "libtp_bench.so"))
    for name in names:
        assert hasattr(bench, name), f"{name} declared in include/tp_bench.h but not exported"
    assert not hasattr(_lib.lib, "tp_bench_fma_peak")
    bench.tp_bench_fma_peak.restype = ctypes.c_int
    bench.tp_bench_fma_peak.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    bench.tp_bench_last_error.restype = ctypes.c_char_p
    assert bench.tp_bench_fma_peak(0, None, None) == _lib.TP_ERR_INVALID_ARG
    assert b"NULL" in bench.tp_bench_last_error()
    assert not hasattr(_lib.lib, "tp_bench_umma_issue")
    bench.tp_bench_umma_issue.restype = ctypes.c_int
    bench.tp_bench_umma_issue.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]
    out = (ctypes.c_double * 2)()
    p0, p1 = ctypes.byref(out, 0), ctypes.byref(out, 8)
    assert bench.tp_bench_umma_issue(64, 1, 0, None, p1, None) == _lib.TP_ERR_INVALID_ARG
    # rejected before any device work: N outside {64, 128, 192, 256}, 3 issuers, too many TMEM columns
    for n, iss, tm in ((96, 1, 0), (64, 3, 0), (256, 4, 0), (256, 2, 1)):
        assert bench.tp_bench_umma_issue(n, iss, tm, p0, p1, None) == _lib.TP_ERR_INVALID_ARG
        assert b"issuers" in bench.tp_bench_last_error()


def test_mesh_validation():
    with pytest.raises(_lib.TPError) as e:
        _lib.tp_mesh_create(0, 4, 4)
    assert e.value.status == _lib.TP_ERR_INVALID_ARG
    with pytest.raises(_lib.TPError):
        _lib.tp_mesh_create(4, 4, 4, -1.0, 1.0, 1.0)
    m = _lib.tp_mesh_create(3, 1, 7, 0.5, 2.0, 1.0)
    _lib.tp_mesh_destroy(m)
    assert _lib.lib.tp_mesh_create(None, 1, 1, 1, 1.0, 1.0, 1.0) == _lib.TP_ERR_INVALID_ARG


def test_operator_argument_validation():
    m = _lib.tp_mesh_create(2, 2, 2)
    try:
        for k in (0, 16):
            with pytest.raises(_lib.TPError) as e:
                _lib.tp_dg_laplace_create(m, k, _lib.TP_FP64)
            assert e.value.status == _lib.TP_ERR_INVALID_ARG
        # degrees 8..15: CUDA-core kernel with FP64 or FP32 vectors only (rejected before any CUDA call)
        for k, p, kern in ((8, _lib.TP_FP16, 1), (15, _lib.TP_BF16, 0), (8, _lib.TP_FP64, 2), (11, _lib.TP_FP32, 2)):
            with pytest.raises(_lib.TPError) as e:
                _lib.tp_dg_laplace_create(m, k, p, kernel=kern)
            assert e.value.status == _lib.TP_ERR_UNSUPPORTED
        # patch-wise kernel: FP64/FP32, k <= 7, at least two cells per direction (checked before any CUDA call)
        for k, p in ((3, _lib.TP_FP16), (2, _lib.TP_BF16), (8, _lib.TP_FP64)):
            with pytest.raises(_lib.TPError) as e:
                _lib.tp_dg_laplace_create(m, k, p, kernel=_lib.TP_KERNEL_PATCH)
            assert e.value.status == _lib.TP_ERR_UNSUPPORTED
        thin = _lib.tp_mesh_create(3, 1, 4)
        try:
            with pytest.raises(_lib.TPError) as e:
                _lib.tp_dg_laplace_create(thin, 3, _lib.TP_FP64, kernel=_lib.TP_KERNEL_PATCH)
            assert e.value.status == _lib.TP_ERR_UNSUPPORTED
        finally:
            _lib.tp_mesh_destroy(thin)
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_dg_laplace_create(m, 3, _lib.TP_FP64, kernel=4)
        assert e.value.status == _lib.TP_ERR_INVALID_ARG
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_dg_laplace_create(m, 3, 9)
        assert e.value.status == _lib.TP_ERR_INVALID_ARG
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_dg_laplace_create(m, 3, _lib.TP_FP64, penalty=5)
        assert e.value.status == _lib.TP_ERR_INVALID_ARG
        # double-word arithmetic: FP64 vectors on the CUDA-core kernel, k <= 7 (checked before any CUDA call)
        for k, p, kern in ((3, _lib.TP_FP32, 0), (3, _lib.TP_FP16, 1), (3, _lib.TP_FP64, 2), (3, _lib.TP_FP64, 3),
                           (8, _lib.TP_FP64, 1)):
            with pytest.raises(_lib.TPError) as e:
                _lib.tp_dg_laplace_create(m, k, p, kernel=kern, dword=1)
            assert e.value.status == _lib.TP_ERR_UNSUPPORTED
            assert "double-word" in _lib.tp_last_error()
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_dg_laplace_create(m, 3, _lib.TP_FP64, dword=2)
        assert e.value.status == _lib.TP_ERR_INVALID_ARG
    finally:
        _lib.tp_mesh_destroy(m)
    assert _lib.lib.tp_apply(None, None, None, None) == _lib.TP_ERR_INVALID_ARG
    assert "NULL" in _lib.tp_last_error()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU failure path")
def test_create_without_gpu_fails_loudly():
    m = _lib.tp_mesh_create(2, 2, 2)
    try:
        with pytest.raises(_lib.TPError) as e:
            _lib.tp_dg_laplace_create(m, 3, _lib.TP_FP64)
        assert e.value.status in (_lib.TP_ERR_CUDA, _lib.TP_ERR_OOM)
    finally:
        _lib.tp_mesh_destroy(m)


def test_failed_operator_creation_releases_mesh_once():
    """A rejected configuration raises TPError and leaves no handle to be freed twice."""
    import gc
    from paper_2407_09621_gb300 import DGLaplace, TPError
    for _ in range(3):
        with pytest.raises(TPError):
            DGLaplace(2, 2, 2, 4, "fp64", kernel=2)  # FP64 tensor kernel: k = 3, 7 only
        gc.collect()


def test_library_resolves_all_of_its_own_symbols():
    """libtp.so must not leave any of its own functions undefined (a shared library links even
    when an internal declaration has no definition; the call would fail only at run time)."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--undefined-only", _lib.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm unavailable")
    undefined = [l.split()[-1] for l in out.stdout.splitlines() if l.strip()]
    own = [u for u in undefined if u.startswith("tp_") or "2tp" in u]
    assert own == []
