"""CPU oracle for the G-NetMon flow-analysis hot path.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the library. It shares no code with the CUDA
path. ``oracle.window`` is the plain definition of one window's per-site result;
``oracle.rmi_ref`` holds the FP64 reference of the learned-index training maths.
"""
from .oracle import *  # noqa: F401,F403
