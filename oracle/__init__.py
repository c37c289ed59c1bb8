"""FP64 CPU oracle for raw C-ToF Gaussian splatting (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
"""
