"""GB300-native semi-implicit PHS-RBF-FD incompressible Navier-Stokes
(Shahane & Vanka, arXiv 2106.07616): CUDA kernels for sm_103a behind a
C-ABI library, with a thin ctypes binding."""
