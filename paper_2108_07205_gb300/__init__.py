"""GB300-native refined-wall Stokes solver (arXiv 2108.07205).

``rwsolve`` is the Python binding of the CUDA library (C ABI in
include/rwsolve.h); ``inputs`` holds the seeded synthetic workloads;
``build`` compiles the library.  Importing the package does not load the
library: ``rwsolve.load()`` does, and raises if it has not been built.
"""
