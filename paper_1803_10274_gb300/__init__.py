"""GB300-native Gaussian-kernel ridge regression through randomized HSS.

Python binding of the C-ABI library ``libkrrhss.so`` (include/krrhss.h):
each function marshals torch CUDA tensors into the C call of the same
name.  All computation runs in the library's CUDA kernels; there is no
CPU or PyTorch fallback.
"""
from .binding import *  # noqa: F401,F403
from .binding import __all__  # noqa: F401
