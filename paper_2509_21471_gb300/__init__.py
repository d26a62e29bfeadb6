"""GB300-native DMK Stokes near-field library (arXiv 2509.21471).

The compute path is the C-ABI shared library built from ``csrc/``; this package
holds its thin ctypes binding (``dmk``) and the seeded input generators
(``workloads``).  Importing ``dmk`` fails loudly if the library was not built.
"""
