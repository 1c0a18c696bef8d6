"""B300-native batched circuit-expectation engine (arXiv 2205.10091 hot path).

The compute path is ``libtc_b300.so`` (CUDA for sm_103a behind a C-ABI,
declared in include/tc.h).  ``paper_2205_10091_b300.native`` is the thin
ctypes binding; importing this package does not load the library, so the
seeded input generators in ``paper_2205_10091_b300.workloads`` can be used
without a GPU.
"""
__all__ = ["workloads"]
