"""GB300-native FP64 solver for the heat and Poisson equations in a closed
cylinder, after the Chebyshev-Chebyshev-Fourier method of arXiv 2206.04827.

The compute path is the C-ABI library ``libcyl.so`` (hand-written CUDA for
sm_103a); ``paper_2206_04827_gb300.cyl`` is its thin ctypes binding and
``paper_2206_04827_gb300.autograd`` the torch.autograd wrapper.  Importing
this package does not load the library; importing ``cyl`` does, and fails
loudly when it has not been built.
"""
