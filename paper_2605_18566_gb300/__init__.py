"""GB300-native (sm_103a) HJ-Gauss frozen-coefficient Picard sweep.

The compute path is libhjg.so (hand-written CUDA, C ABI in include/hjg.h); this package
is its Python binding.  Import fails loudly if the library has not been built.
"""
from ._lib import HJGError, load, symbols  # noqa: F401
from .solver import (Batch, Solver, Surrogate, flock_neighbours, microbench,  # noqa: F401
                     philox_blocks, sample_normals, topology)

__all__ = ["Batch", "Solver", "Surrogate", "HJGError", "flock_neighbours", "microbench", "philox_blocks",
           "sample_normals", "topology", "load", "symbols"]
