"""FP64 CPU oracle for the enhanced MsRSB hot path.

Test infrastructure: only tests/, the smoke check and bench.py's CPU-baseline
leg import this package. It shares no code with the CUDA library.
"""
from . import msrsb  # noqa: F401
