"""FP64 CPU oracle of the half-range lattice Boltzmann Couette solver.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
leg of the benchmark import this package. It shares no code with the CUDA path.
"""
