"""CPU oracle for the RZ PIC-MCC step (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.
"""
from .oracle import Oracle, OracleConfig, philox4x64, philox4x32, boris_move, bfield, node_volume  # noqa: F401
from .oracle import deposit, poisson, efield_at, sigma, sigma_meta, nu_max, field_energy  # noqa: F401
