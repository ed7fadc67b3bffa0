"""FP64 CPU oracle of the lattice Boltzmann inkjet model (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this package; the product path never imports it.
"""
from .oracle import OracleSim, feq, geq, force_term, omega_of_theta, uniform, REC_FIELDS  # noqa: F401
