"""FP64 CPU oracle of the STG wall-modelled MRT-LES lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and by
the benchmark's CPU-baseline / reference leg.  The product path never imports it.
"""
from .oracle import Oracle, OracleConfig, cell_api, load  # noqa: F401
