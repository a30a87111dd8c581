"""FP64 CPU oracle of the MRT lattice Boltzmann hot path.

Test infrastructure only: used by tests/, the smoke check and the
benchmark's CPU-baseline leg, never by the product package.
"""
