"""GB300-native Population Annealing Monte Carlo for Max-Cut (arXiv 2510.21105).

The compute path is the C-ABI library ``libpa.so`` (hand-written CUDA for
sm_103a); ``binding`` is its thin ctypes layer. Importing this package does
not load the library; the first call into ``binding`` does, and raises if the
library has not been built (there is no CPU fallback).
"""
__all__ = ["binding", "workloads", "hexconfig"]
