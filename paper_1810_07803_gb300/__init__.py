"""GB300-native half-range lattice Boltzmann solver for planar Couette flow.

The hot path (the fused WENO-5 / Shakhov / TVD RK-3 time step) is CUDA for
sm_103a behind the C ABI of include/lbc.h; `lbc` is its Python binding.
"""
from .lbc import Batch, LbcError, Solver, equilibrium, quadrature  # noqa: F401
