"""GB300-native free-surface lattice Boltzmann method for liquid-gas-solid flow.

``paper_1712_07028_gb300.lbm`` is the binding of the CUDA library (include/lbm.h; it loads
the library on first use); ``paper_1712_07028_gb300.workloads`` builds the seeded synthetic
bubble-particle columns.
"""
