"""ctypes binding of libtp (include/tp.h): argument marshalling only.

Every function here has the name of the C entry point it calls. Device
vectors are passed as integer addresses (e.g. ``torch.Tensor.data_ptr()``)
and streams as integer ``cudaStream_t`` handles (e.g.
``torch.cuda.current_stream().cuda_stream``). A non-zero tp_status raises
``TPError`` carrying the library's message. There is no fallback: if
libtp.so has not been built, importing this module raises.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtp.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
HEADERS = [os.path.join(INCLUDE, f) for f in ("tp.h", "tp_test.h")]

TP_OK, TP_ERR_INVALID_ARG, TP_ERR_CUDA, TP_ERR_OOM = 0, 1, 2, 3
TP_ERR_NONFINITE, TP_ERR_NOT_CONVERGED, TP_ERR_TIMEOUT, TP_ERR_UNSUPPORTED = 4, 5, 6, 7
STATUS_NAMES = {0: "TP_OK", 1: "TP_ERR_INVALID_ARG", 2: "TP_ERR_CUDA", 3: "TP_ERR_OOM",
                4: "TP_ERR_NONFINITE", 5: "TP_ERR_NOT_CONVERGED", 6: "TP_ERR_TIMEOUT",
                7: "TP_ERR_UNSUPPORTED"}
TP_FP64, TP_FP32, TP_FP16, TP_BF16 = 0, 1, 2, 3
TP_PENALTY_CONFIG, TP_PENALTY_PAPER = 0, 1
TP_KERNEL_AUTO, TP_KERNEL_CUDA_CORE, TP_KERNEL_TENSOR, TP_KERNEL_PATCH = 0, 1, 2, 3


class TPError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libtp.so is not built ({LIB_PATH}); run `python paper_2407_09621_gb300/build.py` "
                      "(the CUDA library is required: there is no CPU fallback)")
lib = ctypes.CDLL(LIB_PATH)


class tp_op_opts(ctypes.Structure):
    _fields_ = [("penalty", ctypes.c_int), ("kernel", ctypes.c_int), ("ec", ctypes.c_int),
                ("tc_type", ctypes.c_int), ("autotune", ctypes.c_int), ("dword", ctypes.c_int)]


class tp_op_info_t(ctypes.Structure):
    _fields_ = [("ncells", ctypes.c_longlong), ("ndofs", ctypes.c_longlong), ("k", ctypes.c_int),
                ("n", ctypes.c_int), ("precision", ctypes.c_int), ("kernel", ctypes.c_int),
                ("elem_bytes", ctypes.c_size_t), ("flops_per_dof", ctypes.c_double),
                ("tensor_path", ctypes.c_int), ("tile_cells", ctypes.c_int), ("approximate", ctypes.c_int),
                ("dword", ctypes.c_int)]


_vp = ctypes.c_void_p
_sig = {
    "tp_last_error": (ctypes.c_char_p, []),
    "tp_mesh_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "tp_mesh_destroy": (ctypes.c_int, [_vp]),
    "tp_dg_laplace_create": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(tp_op_opts)]),
    "tp_op_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(tp_op_info_t)]),
    "tp_op_destroy": (ctypes.c_int, [_vp]),
    "tp_apply": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "tp_apply_host": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_functions(headers=None):
    """Names of every function the given headers (default: include/tp.h) declare."""
    text = ""
    for h in headers or HEADERS:
        with open(h) as f:
            text += f.read()
    return sorted(set(re.findall(r"^\s*(?:tp_status|const char\s*\*|void)\s+(tp_\w+)\s*\(", text, re.M)))


def _check(status):
    if status != TP_OK:
        raise TPError(status, lib.tp_last_error().decode())


def tp_last_error():
    return lib.tp_last_error().decode()


def tp_mesh_create(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0):
    h = _vp()
    _check(lib.tp_mesh_create(ctypes.byref(h), nx, ny, nz, lx, ly, lz))
    return h


def tp_mesh_destroy(mesh):
    _check(lib.tp_mesh_destroy(mesh))


def tp_dg_laplace_create(mesh, k, precision, penalty=TP_PENALTY_CONFIG, kernel=TP_KERNEL_AUTO, ec=0,
                         tc_type=TP_FP16, autotune=0, dword=0):
    h = _vp()
    opts = tp_op_opts(penalty, kernel, ec, tc_type, autotune, dword)
    _check(lib.tp_dg_laplace_create(ctypes.byref(h), mesh, k, precision, ctypes.byref(opts)))
    return h


def tp_op_get_info(op):
    info = tp_op_info_t()
    _check(lib.tp_op_get_info(op, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in tp_op_info_t._fields_}


def tp_op_destroy(op):
    _check(lib.tp_op_destroy(op))


def tp_apply(op, y_ptr, x_ptr, stream=0):
    _check(lib.tp_apply(op, _vp(y_ptr), _vp(x_ptr), _vp(stream)))


def tp_apply_host(op, y_ptr, x_ptr, stream=0):
    _check(lib.tp_apply_host(op, _vp(y_ptr), _vp(x_ptr), _vp(stream)))


# ---------------------------------------------------------------- multigrid / FGMRES
TP_MAX_LEVELS = 16
TP_SMOOTHER_CHEBYSHEV, TP_SMOOTHER_VERTEX_PATCH = 0, 1


class tp_mg_opts(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int), ("ratio", ctypes.c_double), ("safety", ctypes.c_double),
                ("lmax", ctypes.c_double), ("coarse_cells", ctypes.c_int), ("precision", ctypes.c_int),
                ("power_iters", ctypes.c_int), ("kernel", ctypes.c_int), ("ec", ctypes.c_int),
                ("tc_type", ctypes.c_int), ("smoother", ctypes.c_int)]


class tp_mg_info_t(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("precision", ctypes.c_int),
                ("cells", (ctypes.c_int * 3) * TP_MAX_LEVELS), ("ndofs", ctypes.c_longlong * TP_MAX_LEVELS),
                ("lmax", ctypes.c_double * TP_MAX_LEVELS)]


class tp_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("true_rel_residual", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_len", ctypes.c_int),
                ("reorthogonalizations", ctypes.c_int), ("vcycle_graph", ctypes.c_int)]


_sig2 = {
    "tp_mg_create": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, ctypes.POINTER(tp_mg_opts)]),
    "tp_mg_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(tp_mg_info_t)]),
    "tp_mg_level_op": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp)]),
    "tp_mg_destroy": (ctypes.c_int, [_vp]),
    "tp_vcycle": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "tp_mg_smooth": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "tp_mg_restrict": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "tp_mg_prolongate_add": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "tp_mg_coarse_solve": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "tp_fgmres_create": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, _vp, ctypes.c_int]),
    "tp_fgmres_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(tp_solve_info), _vp]),
    "tp_solver_destroy": (ctypes.c_int, [_vp]),
}
for _name, (_res, _args) in _sig2.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def tp_mg_create(op, degree=3, ratio=15.0, safety=1.1, lmax=0.0, coarse_cells=4, precision=TP_FP32,
                 power_iters=20, kernel=TP_KERNEL_CUDA_CORE, ec=0, tc_type=TP_FP16, smoother=TP_SMOOTHER_CHEBYSHEV):
    h = _vp()
    o = tp_mg_opts(degree, ratio, safety, lmax, coarse_cells, precision, power_iters, kernel, ec, tc_type, smoother)
    _check(lib.tp_mg_create(ctypes.byref(h), op, ctypes.byref(o)))
    return h


def tp_mg_get_info(mg):
    info = tp_mg_info_t()
    _check(lib.tp_mg_get_info(mg, ctypes.byref(info)))
    L = info.levels
    return {"levels": L, "precision": info.precision,
            "cells": [tuple(info.cells[l]) for l in range(L)], "ndofs": [info.ndofs[l] for l in range(L)],
            "lmax": [info.lmax[l] for l in range(L)]}


def tp_mg_level_op(mg, level):
    h = _vp()
    _check(lib.tp_mg_level_op(mg, level, ctypes.byref(h)))
    return h


def tp_mg_destroy(mg):
    _check(lib.tp_mg_destroy(mg))


def tp_vcycle(mg, x_ptr, b_ptr, stream=0):
    _check(lib.tp_vcycle(mg, _vp(x_ptr), _vp(b_ptr), _vp(stream)))


def tp_mg_smooth(mg, level, x_ptr, b_ptr, stream=0):
    _check(lib.tp_mg_smooth(mg, level, _vp(x_ptr), _vp(b_ptr), _vp(stream)))


def tp_mg_restrict(mg, level, coarse_ptr, fine_ptr, stream=0):
    _check(lib.tp_mg_restrict(mg, level, _vp(coarse_ptr), _vp(fine_ptr), _vp(stream)))


def tp_mg_prolongate_add(mg, level, fine_ptr, coarse_ptr, stream=0):
    _check(lib.tp_mg_prolongate_add(mg, level, _vp(fine_ptr), _vp(coarse_ptr), _vp(stream)))


def tp_mg_coarse_solve(mg, x_ptr, b_ptr, stream=0):
    _check(lib.tp_mg_coarse_solve(mg, _vp(x_ptr), _vp(b_ptr), _vp(stream)))


def tp_fgmres_create(op, mg=None, restart=30):
    h = _vp()
    _check(lib.tp_fgmres_create(ctypes.byref(h), op, mg, restart))
    return h


def tp_fgmres_solve(solver, x_ptr, b_ptr, rtol=1e-10, maxit=200, stream=0, raise_on_error=True):
    """Returns (status, info dict); raises TPError on failure unless raise_on_error is False."""
    info = tp_solve_info()
    st = lib.tp_fgmres_solve(solver, _vp(x_ptr), _vp(b_ptr), rtol, maxit, ctypes.byref(info), _vp(stream))
    d = {"iterations": info.iterations, "restarts": info.restarts, "converged": info.converged,
         "rel_residual": info.rel_residual, "true_rel_residual": info.true_rel_residual,
         "history": [info.history[i] for i in range(info.history_len)] if info.history else [],
         "reorthogonalizations": info.reorthogonalizations, "vcycle_graph": info.vcycle_graph}
    if st != TP_OK and raise_on_error:
        raise TPError(st, lib.tp_last_error().decode())
    return st, d


def tp_solver_destroy(solver):
    _check(lib.tp_solver_destroy(solver))


# ---------------------------------------------------------------- host apply without device allocation
TP_NOALLOC_MAX_BYTES = 8 * 1024 * 1024
lib.tp_apply_host_noalloc.restype = ctypes.c_int
lib.tp_apply_host_noalloc.argtypes = [_vp, _vp, _vp, _vp]


def tp_apply_host_noalloc(op, y_ptr, x_ptr, stream=0):
    _check(lib.tp_apply_host_noalloc(op, _vp(y_ptr), _vp(x_ptr), _vp(stream)))


lib.tp_op_check.restype = ctypes.c_int
lib.tp_op_check.argtypes = [_vp]


def tp_op_check(op):
    _check(lib.tp_op_check(op))


lib.tp_test_set_wait_fault.restype = ctypes.c_int
lib.tp_test_set_wait_fault.argtypes = [_vp, ctypes.c_int, ctypes.c_double]


def tp_test_set_wait_fault(op, withhold_first_copy, wait_limit_s):
    """Failure-injection hook of include/tp_test.h (tests of the bounded device waits only)."""
    _check(lib.tp_test_set_wait_fault(op, int(withhold_first_copy), float(wait_limit_s)))


lib.tp_batch_solve_solvers.restype = ctypes.c_int
lib.tp_batch_solve_solvers.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp]


def tp_batch_solve_solvers(solvers, x_ptrs, b_ptrs, rtol=1e-10, maxit=300, streams=8):
    """Concurrent solves of the caller's (solver, x, b) entries; returns (infos, statuses, seconds)."""
    n = len(solvers)
    if not (n == len(x_ptrs) == len(b_ptrs)):
        raise ValueError("solvers, x_ptrs and b_ptrs must have the same length")
    sv = (_vp * n)(*[s if isinstance(s, _vp) else _vp(s) for s in solvers])
    xv = (_vp * n)(*[_vp(p) for p in x_ptrs])
    bv = (_vp * n)(*[_vp(p) for p in b_ptrs])
    opts = tp_batch_opts(TP_FP32, TP_KERNEL_CUDA_CORE, 0, 30, rtol, maxit, streams, 0, TP_SMOOTHER_CHEBYSHEV)
    infos = (tp_solve_info * n)()
    sts = (ctypes.c_int * n)()
    total = ctypes.c_double()
    _check(lib.tp_batch_solve_solvers(sv, xv, bv, n, ctypes.byref(opts), infos, sts, ctypes.byref(total)))
    out = [{"iterations": i.iterations, "converged": i.converged, "rel_residual": i.rel_residual,
            "true_rel_residual": i.true_rel_residual} for i in infos]
    return out, list(sts), total.value


# ---------------------------------------------------------------- Poisson problem data
lib.tp_rhs_sines.restype = ctypes.c_int
lib.tp_rhs_sines.argtypes = [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), _vp]
lib.tp_l2_error_sines.restype = ctypes.c_int
lib.tp_l2_error_sines.argtypes = [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), _vp]


def _modes_arrays(modes):
    a = (ctypes.c_double * len(modes))(*[float(m[0]) for m in modes])
    pqr = (ctypes.c_int * (3 * len(modes)))(*[int(v) for m in modes for v in m[1:4]])
    return a, pqr


def tp_rhs_sines(op, b_ptr, modes=((1.0, 1, 1, 1),), stream=0):
    """modes: sequence of (a, p, q, r)."""
    a, pqr = _modes_arrays(modes)
    _check(lib.tp_rhs_sines(op, _vp(b_ptr), len(modes), a, pqr, _vp(stream)))


def tp_l2_error_sines(op, u_ptr, modes=((1.0, 1, 1, 1),), stream=0):
    a, pqr = _modes_arrays(modes)
    out = ctypes.c_double()
    _check(lib.tp_l2_error_sines(op, _vp(u_ptr), len(modes), a, pqr, ctypes.byref(out), _vp(stream)))
    return out.value


# ---------------------------------------------------------------- batched solves
class tp_batch_problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("k", ctypes.c_int),
                ("nmodes", ctypes.c_int), ("a", ctypes.POINTER(ctypes.c_double)),
                ("pqr", ctypes.POINTER(ctypes.c_int)), ("x", _vp)]


class tp_batch_opts(ctypes.Structure):
    _fields_ = [("mg_precision", ctypes.c_int), ("kernel", ctypes.c_int), ("ec", ctypes.c_int),
                ("restart", ctypes.c_int), ("rtol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("streams", ctypes.c_int), ("autotune", ctypes.c_int), ("smoother", ctypes.c_int)]


class tp_batch_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("l2_error", ctypes.c_double),
                ("seconds", ctypes.c_double)]


lib.tp_batch_solve.restype = ctypes.c_int
lib.tp_batch_solve.argtypes = [ctypes.POINTER(tp_batch_problem), ctypes.c_int, ctypes.POINTER(tp_batch_opts),
                               ctypes.POINTER(tp_batch_result), ctypes.POINTER(ctypes.c_double)]


def tp_batch_solve(problems, mg_precision=TP_FP32, kernel=TP_KERNEL_CUDA_CORE, ec=0, restart=30, rtol=1e-10,
                   maxit=300, streams=8, autotune=0, smoother=TP_SMOOTHER_CHEBYSHEV):
    """problems: list of dicts {cells: (nx, ny, nz) or int, k, modes: [(a, p, q, r), ...], x_ptr (optional)}.
    Returns (list of result dicts, total solve seconds)."""
    n = len(problems)
    arr = (tp_batch_problem * n)()
    keep = []
    for i, p in enumerate(problems):
        c = p["cells"]
        nx, ny, nz = (c, c, c) if isinstance(c, int) else c
        a, pqr = _modes_arrays(p["modes"])
        keep += [a, pqr]
        arr[i] = tp_batch_problem(nx, ny, nz, p["k"], len(p["modes"]), a, pqr, _vp(p.get("x_ptr") or 0))
    opts = tp_batch_opts(mg_precision, kernel, ec, restart, rtol, maxit, streams, autotune, smoother)
    res = (tp_batch_result * n)()
    total = ctypes.c_double()
    _check(lib.tp_batch_solve(arr, n, ctypes.byref(opts), res, ctypes.byref(total)))
    out = [{f: getattr(r, f) for f, _ in tp_batch_result._fields_} for r in res]
    return out, total.value
