"""CPU FP64 oracle for the QTT Fokker-Planck path.

TEST INFRASTRUCTURE ONLY: imported by tests, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py.  The product library never uses it.
"""
from .fd import *  # noqa: F401,F403
