"""GB300-native state-vector emulation of the hybrid VQE + DBBSC hot path (arXiv:2405.11567).

The compute path is the C-ABI library built from ``csrc/`` (hand-written CUDA
for sm_103a); :mod:`.sv` is its thin ctypes binding and :mod:`.autograd` wraps
energy + adjoint gradient as a ``torch.autograd.Function``.  Importing the
package loads nothing; the shared library is opened on first use and a missing
library is an error, never a fallback.
"""
