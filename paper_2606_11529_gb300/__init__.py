"""GB300-native (sm_103a) 3D Gaussian Splatting tile-splatting path.

The compute runs in the hand-written CUDA library ``libxpr.so`` (C ABI in
``include/xpr.h``); ``binding`` marshals arguments to it, ``render`` wraps the
path in a ``torch.autograd.Function``.  Importing the package does not load
the library; the first call that needs it does, and fails loudly if it is
missing.
"""
__all__ = ["scenes"]
