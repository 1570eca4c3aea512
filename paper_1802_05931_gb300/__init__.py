"""GB300-native driven-dissipative quantum Monte Carlo (arXiv:1802.05931).

The DDQMC step runs in hand-written CUDA kernels for sm_103a behind the C-ABI
of ``libddqmc.so`` (declared in ``include/ddqmc.h``); ``ddqmc`` is the thin
ctypes binding with the same names.
"""
from .ddqmc import DDQMCError, Run, load  # noqa: F401
