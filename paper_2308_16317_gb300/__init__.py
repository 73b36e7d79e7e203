"""GB300-native LSMS tau_00 library (arXiv 2308.16317 hot path).

The compute path lives in the C-ABI shared library built from ``csrc/``
(``libmust.so``); ``binding`` marshals arguments to it with ctypes.  Importing
this package does not load the library; ``binding.load()`` does, and fails
loudly if it has not been built.
"""
__all__ = ["binding", "workload"]
