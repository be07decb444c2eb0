"""FP64 CPU oracle of the GEA pressure-based Euler time step.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline leg may import this package. The CUDA library never uses it.
"""
from .oracle import (  # noqa: F401
    Oracle, OracleState, build_oracle, set_reverse_sums, READING_K_LAGGED, BC_EVEN, BC_U, BC_W, BC_H,
)
