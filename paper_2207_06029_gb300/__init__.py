"""GB300-native lattice-Boltzmann / dynamic immersed-boundary solver (arXiv 2207.06029).

The compute path is the CUDA library ``liblbib.so`` (C ABI declared in
``include/lbib.h``); ``paper_2207_06029_gb300.lbib`` is its ctypes binding.
Importing this package loads nothing; the binding loads the library on first use.
"""
