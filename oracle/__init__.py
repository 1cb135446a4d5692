"""FP64 CPU oracle for the ReLCP hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the library.  It shares no code
with the CUDA path; see relcp_oracle.py (Algorithm 1 of the paper) and
oracle.c (pairs, SNSD, Lemke).
"""
from . import relcp_oracle  # noqa: F401
