"""CPU oracle for the multi-MSB replacement RDHEI method (arXiv 2302.07992).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; the product package never imports it.  The
arithmetic of the method lives in ``rdhei_oracle.c`` (plain C, literal paper steps),
which this package compiles and calls through ctypes; the security and quality
statistics of Sec. IV-C are written out in fp64 numpy in ``metrics.py``.
"""
from .oracle import *  # noqa: F401,F403
