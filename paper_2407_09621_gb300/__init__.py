"""GB300-native sum-factorized SIPG DG-Laplace apply and mixed-precision
multigrid/FGMRES Poisson solve (Cui, "Acceleration of Tensor-Product
Operations with Tensor Cores").

The compute path is libtp.so (CUDA for sm_103a, C ABI in include/tp.h).
This package only marshals arguments to it; see ``_lib`` for the binding
and ``ops`` for small conveniences over torch tensors.
"""
from . import _lib  # noqa: F401  (raises if libtp.so is missing)
from ._lib import *  # noqa: F401,F403
from .ops import DGLaplace, PRECISIONS  # noqa: F401
