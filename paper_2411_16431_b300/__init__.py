"""sgtn: B300-native tensor-network branch-and-bound for Ising spin glasses (arXiv:2411.16431).

``lattices`` draws seeded instances; ``sgtn`` is the thin binding of the CUDA
library ``libsgtn.so`` (C ABI in include/sgtn.h).  Importing the package does
not load the library; ``sgtn.load()`` does, and raises if it is missing.
"""
