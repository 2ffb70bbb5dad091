"""GB300-native library for the high-order LDG thermosphere model (arXiv 2306.01085).

Submodules: workloads (seeded inputs), build (nvcc build of libdg_gb300.so), dg (ctypes binding of
include/dg.h). Importing the package loads nothing; the CUDA library is loaded on first use.
"""
