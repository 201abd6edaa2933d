"""Plain FP64 CPU oracle for the quadrature-free DG shallow-water scheme.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and
the CPU-baseline leg of the benchmark, never by the library.
"""
from .oracle import Oracle, build_oracle, build_variant, ms_point, source  # noqa: F401
