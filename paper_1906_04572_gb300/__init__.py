"""GB300 (sm_103a) implementation of Compressed Randomized UTV (CoR-UTV) with
the power method and of ALM-CoRUTV robust PCA (Kaloorazi & de Lamare).

The compute path is libcorutv.so (CUDA kernels behind the C ABI of
include/corutv.h); `corutv` is its ctypes binding and `build` compiles it.
"""

from . import corutv  # noqa: F401
from .corutv import Context, CorutvError  # noqa: F401
