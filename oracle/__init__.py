"""CPU oracle for the HFX force/stress hot path (TEST INFRASTRUCTURE ONLY).

Only tests, the package smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA path.
"""
from .hfx_oracle import Options, OraclePlan, Result, evaluate  # noqa: F401
