"""Seeded synthetic inputs (G0 tables, cluster geometry, chain parameters).

Shared by the CUDA path, its tests, the benchmark and the oracle.  It holds no
part of the submatrix-update arithmetic.
"""
from . import g0tables, configs  # noqa: F401
