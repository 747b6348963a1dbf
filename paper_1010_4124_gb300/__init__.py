"""GB300-native finite-difference lattice Boltzmann step (D2V19 + WENO5).

The compute path is the C-ABI library libklb.so (hand-written CUDA for
sm_103a, declared in include/klb.h); `paper_1010_4124_gb300.klb` is its thin
ctypes binding.  Importing this package does not load the library; the first
use of `klb` does, and fails loudly if it has not been built.
"""
__all__ = ["inputs", "klb"]
