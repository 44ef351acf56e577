"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package holds no arithmetic of the MsRSB method itself: it builds fine-scale
operators A and right-hand sides b (finite-volume Darcy, Q1 elasticity), random
coefficient fields and grid descriptions. Both sides of every parity test receive
the same (A, b) from here, so discretisation details never enter parity.
"""
from .fields import gaussian_random_field, rotation_zyx, rotation_2d  # noqa: F401
from .darcy import mpfa_o, tpfa, darcy_2d_case, darcy_3d_case  # noqa: F401
from .elastic import q1_elasticity, elastic_3d_case  # noqa: F401
from .grid import Grid  # noqa: F401
