"""CPU oracle for the multi-MSB replacement RDHEI method (arXiv 2302.07992).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; the product package never imports it.  The
arithmetic lives in ``rdhei_oracle.c`` (plain C, literal paper steps); this package
only compiles it and marshals numpy arrays through ctypes.
"""
from .oracle import *  # noqa: F401,F403
