"""GB300 (sm_103a) temporally blocked 3D 7-point Jacobi library.

``jacobi`` binds the C ABI of libjacobi.so (include/jacobi.h); ``inputs``
holds the seeded synthetic workloads; ``build`` compiles the CUDA sources.
Importing the package loads nothing: the CUDA library is loaded on the first
call and every call fails loudly if it is missing.
"""
__all__ = ["jacobi", "inputs", "build"]
