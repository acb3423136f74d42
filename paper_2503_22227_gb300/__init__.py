"""GB300-native RNS hot path for CKKS / BFV / BGV (homomorphic multiply with
relinearisation, rotation, rescale / modulus switch), after the CAT
framework (arXiv 2503.22227).

The compute path is the C-ABI library ``libcatfhe.so`` (hand-written CUDA
for sm_103a); :mod:`.api` is a thin ctypes binding over it.  Importing this
package does not load the library; :func:`api.load` does, and raises if it
is missing.
"""

__all__ = ["api", "workloads"]
