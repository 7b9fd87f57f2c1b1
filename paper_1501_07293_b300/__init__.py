"""B300-native finite-difference micromagnetic solver (arXiv:1501.07293 hot path).

The compute path is the C-ABI library ``libmm_b300.so`` (hand-written sm_103a
CUDA kernels); ``solver`` is a thin ctypes binding over it.  Importing this
package does not load the library; ``solver`` does, and fails loudly when it
is missing.
"""
__version__ = "0.1.0"
