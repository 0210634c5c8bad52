"""B300-native (sm_103a) implementation of the matrix-free T-matrix
multiple-scattering method of arXiv 2107.09879 (GMRES forward and adjoint
solves, sub-region decomposition). The compute path is the native library
libtmat.so (include/tmat.h); `_lib` is its ctypes binding."""
