"""GB300-native carousel phase retrieval (CPRA, arXiv 2402.05283) hot path.

The compute lives in ``libcpra.so`` (hand-written sm_103a CUDA kernels behind
the C ABI of ``include/cpra.h``); this package is its ctypes binding.
"""
from .binding import *  # noqa: F401,F403
from .binding import Plan, Batch, Server, make_config, lib, CpraError  # noqa: F401
