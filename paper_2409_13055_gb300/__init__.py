"""GB300-native differentiable tile-based 3D Gaussian Splatting mapping step.

The compute path lives in ``libgs_gb300.so`` (hand-written CUDA for sm_103a,
built from ``csrc/``) behind the C-ABI declared in ``include/gs.h``.  This
package adds the thin ctypes binding (``binding``), the autograd wrapper and
mapping-iteration driver (``mapping``), and seeded synthetic workloads
(``scenes``).  Importing the package loads nothing; the CUDA library is loaded
on first use and its absence is an error, never a fallback.
"""
__all__ = ["scenes"]
