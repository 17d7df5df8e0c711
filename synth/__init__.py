"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This package holds workload descriptions only: shape parameters drawn from
seeded generators, wavenumbers, discretisation sizes and incident directions.
It contains none of the method's arithmetic (no geometry, no kernels, no
solves); both the product and the oracle import it and nothing else in common.
"""
from .workloads import *  # noqa: F401,F403
