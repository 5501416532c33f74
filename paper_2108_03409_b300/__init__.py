"""B300-native NQS variational Monte Carlo hot path (arXiv:2108.03409, jVMC).

The compute path is the C-ABI library ``libvmc.so`` (hand-written sm_103a CUDA kernels,
declared in ``include/vmc.h``).  ``paper_2108_03409_b300.vmc`` is the thin ctypes binding
with the same entry-point names; ``paper_2108_03409_b300.inputs`` draws the seeded
synthetic inputs.  Importing this package does not load the native library; the binding
loads it on first use and raises if it is missing.
"""
__all__ = ["inputs", "vmc"]
