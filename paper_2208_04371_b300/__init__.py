"""B300-native Yee FDTD transmission-line S-parameter library (arXiv 2208.04371).

Submodules:
  yf          ctypes binding of the CUDA library libyeefdtd.so (include/yeefdtd.h)
  workloads   seeded synthetic microstrip inputs
  build       nvcc build of the library for sm_103a

Importing the package loads nothing; `from paper_2208_04371_b300 import yf` loads the
compiled library and fails if it has not been built.
"""
