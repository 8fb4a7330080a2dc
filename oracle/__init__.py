"""FP64 CPU oracle for the AdpSplit hot path.

Test infrastructure only: the test suite, the smoke check and the CPU-baseline leg
of the benchmark are the only users. It shares no code with the CUDA path.
"""
from .oracle import *  # noqa: F401,F403
