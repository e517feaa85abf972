"""GB300 (sm_103a) batched space-time Extend for ST-pRRTC.

The compute path is the CUDA library built from csrc/ (C ABI: include/stp.h);
``stp`` is its thin ctypes binding.
"""
from . import stp  # noqa: F401
from .stp import Problem, StpError, problem_from  # noqa: F401
