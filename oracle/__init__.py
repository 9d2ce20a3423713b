"""CPU oracle for the SoA particle hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
package.  It shares no code with the CUDA library (paper_1710_03462_b300) and never
imports it.  See soax_oracle.c for what each function computes and where it comes
from; the pins that tie it to the paper and to mathematics live in tests/test_oracle_*.
"""
from .oracle import *  # noqa: F401,F403
