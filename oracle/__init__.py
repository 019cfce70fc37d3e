"""Plain FP64 CPU oracle of the DEC steady-conduction hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call,
link or execute this package: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference leg use it.  It shares no code,
table or helper with the CUDA library; the two see the same seeded inputs
from ``dec_inputs`` and nothing else.

Every function follows one passage of the paper (arXiv 2104.05999), cited in
its docstring, and is written as the definition it implements: no blocking,
fusion or reordering beyond that definition.  numpy / scipy serve as library
primitives (small dense solves, sparse matrix-vector products, sorting).
"""
from .dec import *          # noqa: F401,F403
from .dec import __all__    # noqa: F401
