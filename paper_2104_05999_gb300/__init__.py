"""GB300-native DEC steady-conduction path (arXiv 2104.05999).

The computation lives in the CUDA library ``lib/libdec_gb300.so`` (sources
under ``csrc/``, C declarations in ``include/dec.h``); ``abi`` is its ctypes
binding and ``run`` strings the entry points together for a whole solve.
"""
from . import abi
from .abi import Context, DecError
from .run import run_path, PathResult

__all__ = ["abi", "Context", "DecError", "run_path", "PathResult"]
