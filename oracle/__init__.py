"""FP64 CPU oracle for backward RK4 tracing of Kerr null geodesics.

Test infrastructure only: the parity reference for the CUDA tracer.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library and imports nothing from it.
"""
from .oracle import *  # noqa: F401,F403
