"""GB300-native multicomponent lattice Boltzmann step (Stefan-Maxwell species +
compressible momentum/energy lattices on D3Q27), after Sawant, Dorschner &
Karlin, arXiv 2004.11286.

The compute path lives in the CUDA shared library ``liblbm_mix.so`` built from
``csrc/``; ``binding`` is a thin ctypes layer over its C ABI
(``include/lbm_mix.h``).  Importing this package does not load the library;
the first call that needs it does, and fails loudly if it is missing.
"""

__all__ = ["binding", "workloads"]
