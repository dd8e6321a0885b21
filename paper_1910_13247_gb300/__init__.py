"""GB300-native matrix-free Q_k Laplacian (vmult, CG, Chebyshev, mixed precision).

The compute path is the CUDA library ``libmfx.so`` (C-ABI declared in
``include/mfx.h``); :mod:`paper_1910_13247_gb300.mfx` is its thin ctypes
binding.  The library is loaded on first use; if it is missing the binding
raises instead of falling back to any CPU path.
"""
__all__ = ["mfx", "synthetic"]
