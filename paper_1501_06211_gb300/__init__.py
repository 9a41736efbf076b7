"""GB300-native domain-decomposition solver for linear elasticity in topology
optimisation (Turner, Kocvara, Loghin, arXiv:1501.06211).

The compute path is libddel.so (CUDA, sm_103a) behind the C ABI of
include/ddel.h; ``paper_1501_06211_gb300.ddel`` is its ctypes binding.
"""
from .build import build, LIB  # noqa: F401
