"""Shared helpers of the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import torch

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 5e-3, "bf16": 5e-3}
DTYPES = {"fp64": torch.float64, "fp32": torch.float32, "fp16": torch.float16, "bf16": torch.bfloat16}


def rel_l2(v, ref):
    """Relative l2 error of Sec. 5.2: ||v - v_ref||_2 / ||v_ref||_2."""
    v = np.asarray(v, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(v - ref) / np.linalg.norm(ref))


def to_device(x64, prec):
    """Round an FP64 host vector to the operator's storage type on the GPU."""
    return torch.from_numpy(x64).to(device="cuda", dtype=DTYPES[prec])


def to_host64(t):
    return t.to(torch.float64).cpu().numpy()
