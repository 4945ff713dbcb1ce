"""GB300-native exact 1-NN DTW search with the LB_Enhanced^V lower bound
(Tan, Petitjean, Webb, arXiv 1808.09617).

The compute path is the CUDA library ``libnndtw.so`` (built in-tree by
``paper_1808_09617_gb300.build``) behind a C ABI declared in
``include/nndtw.h``; ``paper_1808_09617_gb300.nndtw`` is its thin Python
binding.  Importing this package does not load the library; the first call
into the binding does, and raises if the library is missing.
"""
__all__ = ["nndtw", "synth", "build"]
