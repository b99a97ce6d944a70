"""GB300-native element-model N-body library (arXiv:2303.12166).

The compute path is libnbody.so (hand-written CUDA for sm_103a behind the C
ABI of include/nbody.h); :mod:`paper_2303_12166_gb300.nbody` is its ctypes
binding.  Build the library with ``python -m paper_2303_12166_gb300.build``.
"""
