"""CPU FP64 oracle for HPS leaf condensation (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg use it; the
GPU library never imports it.
"""
from .hps_oracle import *  # noqa: F401,F403
