"""GB300-native matrix renewal convolution: FFT-Newton inversion of A = e0 - q.

The compute path is the C-ABI library ``libmrc.so`` (hand-written sm_103a CUDA
kernels); ``paper_2605_30379_gb300.mrc`` is a thin ctypes binding over it that
marshals torch CUDA tensors.  ``synth`` builds seeded synthetic inputs.
Importing the package does not load the CUDA library; the first call into
``mrc`` does, and fails loudly if it has not been built.
"""
__all__ = ["mrc", "synth"]
