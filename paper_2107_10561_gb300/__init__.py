"""GB300-native space-time multigrid (dG(k) x Q2/P1disc Navier-Stokes slabs) behind the libstm C-ABI.

The compute path is libstm.so (hand-written CUDA for sm_103a, built by `build.py`); this package
holds only its ctypes binding (`solver`) and the autograd wrapper of the adjoint solve.
"""
from .solver import Hierarchy, make_params  # noqa: F401
