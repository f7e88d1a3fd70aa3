"""A-orthonormal thin QR by modified Gram-Schmidt on GB300 (sm_103a).

GB300-native implementation of the hot path of Imakura & Yamamoto,
"Efficient implementations of the modified Gram-Schmidt orthogonalization
with a non-standard inner product" (arXiv 1703.10440): Z = QR with
Q^T A Q = I for sparse SPD A, in the naive 2n-MV form and the paper's
n-MV MGS-HA and MGS-HP forms.

The computation lives in ``libmgsa.so`` (CUDA C++, C-ABI declared in
``include/mgsa.h``); :mod:`.mgsa` is its ctypes binding.
"""
from . import mgsa  # noqa: F401
from .mgsa import Handle, MgsaError, VARIANTS  # noqa: F401

__all__ = ["mgsa", "Handle", "MgsaError", "VARIANTS"]
