"""FP64 CPU oracle for the H-matrix hot path of arXiv:1706.09384.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product package never imports
it, and it shares no code with the CUDA path.  See ``oracle.c`` for the
algorithms and their citations.
"""
from .oracle import *  # noqa: F401,F403
