"""GB300-native pseudopotential MRT lattice Boltzmann step (D2Q9) with the original and
the improved third-order source term of Huang, Huang & Li (2026).

The compute path is the CUDA library built from csrc/ (C ABI declared in include/lbm.h);
`lbm` is its thin ctypes binding and loads it on first use, failing loudly when the
library has not been built.  `inputs` holds the seeded synthetic input generators.
"""
__all__ = ["lbm", "inputs"]
