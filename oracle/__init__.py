"""FP64 CPU oracle of the lattice Boltzmann inkjet model (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this package; the product path never imports it.
"""
from .oracle import OracleSim, OracleSim3, feq, feq3, force_term, force_term3, geq, geq3, lattice3, omega_of_theta, set_threads, threads, uniform, REC_FIELDS  # noqa: F401
