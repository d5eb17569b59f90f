"""GB300 (sm_103a) multigrid-preconditioned FGMRES solver for the condensed
momentum system of a monolithic Newton-multigrid FSI method.

The compute lives in libnmg.so (CUDA, C ABI in include/nmg.h); ``nmg`` is its
ctypes binding and ``session`` a small convenience layer that uploads a level
hierarchy and calls the library.
"""
