"""GB300 (sm_103a) hot path of the Schwarz-preconditioned two-flavour Wilson
HMC with a one-dimensional (x0-slab) domain decomposition (Hasenbusch,
Lattice 2007).

The product is ``liblqcd.so`` (C-ABI: include/lqcd.h); ``lqcd`` is its thin
Python binding and ``synthetic`` the seeded input generator.
"""
__all__ = ["lqcd", "synthetic"]
