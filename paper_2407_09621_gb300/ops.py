"""Convenience wrapper over the C ABI for callers holding torch tensors.

Marshalling only: pointers, sizes and stream handles are passed to libtp;
no arithmetic of the method happens here.
"""
import torch

from . import _lib

PRECISIONS = {
    "fp64": (_lib.TP_FP64, torch.float64),
    "fp32": (_lib.TP_FP32, torch.float32),
    "fp16": (_lib.TP_FP16, torch.float16),
    "bf16": (_lib.TP_BF16, torch.bfloat16),
}


class DGLaplace:
    """SIPG Laplace operator of degree k on an nx*ny*nz box mesh (owns its handles)."""

    def __init__(self, nx, ny, nz, k, precision="fp64", penalty=_lib.TP_PENALTY_CONFIG,
                 kernel=_lib.TP_KERNEL_AUTO, ec=0, lengths=(1.0, 1.0, 1.0), tc_type=_lib.TP_FP16, autotune=0,
                 dword=0):
        self.op = self.mesh = None
        self.prec, self.dtype = PRECISIONS[precision]
        self.mesh = _lib.tp_mesh_create(nx, ny, nz, *lengths)
        try:
            self.op = _lib.tp_dg_laplace_create(self.mesh, k, self.prec, penalty, kernel, ec, tc_type, autotune,
                                                dword)
        except Exception:
            mesh, self.mesh = self.mesh, None
            _lib.tp_mesh_destroy(mesh)
            raise
        self.info = _lib.tp_op_get_info(self.op)
        self.ndofs = self.info["ndofs"]

    def apply(self, y, x, stream=None):
        """y = A x for device tensors of the operator's dtype (contiguous, ndofs entries)."""
        for t in (x, y):
            if t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != self.ndofs:
                raise ValueError("x and y must be contiguous CUDA tensors of the operator's dtype and size")
        s = stream if stream is not None else torch.cuda.current_stream()
        _lib.tp_apply(self.op, y.data_ptr(), x.data_ptr(), s.cuda_stream)
        return y

    def apply_host(self, y, x, stream=None):
        """y = A x for host tensors (copies inside the call)."""
        for t in (x, y):
            if t.dtype != self.dtype or t.is_cuda or not t.is_contiguous() or t.numel() != self.ndofs:
                raise ValueError("x and y must be contiguous host tensors of the operator's dtype and size")
        s = stream.cuda_stream if stream is not None else 0
        _lib.tp_apply_host(self.op, y.data_ptr(), x.data_ptr(), s)
        return y

    def check(self):
        """Synchronize and raise TPError if a bounded device wait of this operator gave up."""
        _lib.tp_op_check(self.op)

    def close(self):
        if getattr(self, "op", None):
            _lib.tp_op_destroy(self.op)
            self.op = None
        if getattr(self, "mesh", None):
            _lib.tp_mesh_destroy(self.mesh)
            self.mesh = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
