"""GB300-native differentiable raw C-ToF Gaussian splatting (arXiv 2505.05356).

The compute path is the C-ABI library ``libgftorf.so`` (hand-written sm_103a
CUDA); ``gftorf`` is its thin ctypes binding and ``RenderCToF`` the autograd
wrapper.  Importing this package does not load the library; the first call
into ``gftorf`` does, and raises if it is missing.
"""
