"""ML(n)BiCGStab on GB300 (sm_103a): a CUDA library with a C ABI
(include/mlbicgstab.h) and its Python binding.

Submodules
    mlbicgstab  ctypes binding with the C entry-point names
    workloads   seeded synthetic linear systems (inputs only)
    build       in-tree nvcc build of libmlbicgstab.so

Importing the package does not load the CUDA library; the binding loads it
on first use and raises if it is missing.
"""
