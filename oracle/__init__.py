"""Oracle for the homogeneous-medium RTE Fredholm operators.

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 CPU code that evaluates what the
fast method computes straight from its definition (direct Nystrom sums, dense
solves, a textbook GMRES).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  The product package never
imports it, and it imports nothing from the product package.

Parity status per function is listed in ``oracle/core.py`` (homogeneous medium)
and ``oracle/inhom.py`` (the inhomogeneous-medium direct Nystrom matrix).
"""
from .core import *  # noqa: F401,F403
