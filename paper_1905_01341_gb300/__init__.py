"""GB300-native FMM-accelerated boundary-element library for bubble dynamics
(arXiv:1905.01341): CUDA kernels for sm_103a behind the C ABI of include/bem.h, with a thin
ctypes binding (``bem``)."""
from . import bem  # noqa: F401
from .bem import BemContext, BemError  # noqa: F401
