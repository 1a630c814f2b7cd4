"""paper_1704_08657_gb300 -- non-separable lifting 2-D DWT on GB300.

The library is ``libdwt2.so`` (C ABI in ``include/dwt2.h``), built in-tree by
``paper_1704_08657_gb300.build``.  ``abi`` is the ctypes binding with the same
names; ``dwt`` adds PyTorch helpers (plans over CUDA tensors, autograd);
``synth`` holds the seeded synthetic input recipes.
"""
__all__ = ["abi", "dwt", "synth", "build"]
