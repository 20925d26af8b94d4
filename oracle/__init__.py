"""CPU oracle for the Lanczos GW hot path (test infrastructure only).

Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark import this package; the library never does.
"""
from .gw_oracle import *  # noqa: F401,F403
