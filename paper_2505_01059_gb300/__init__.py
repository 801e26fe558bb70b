"""GB300-native Model Tensor Planning hot path (arXiv 2505.01059).

The compute lives in ``libmtp.so`` (hand-written CUDA for sm_103a behind the C
ABI of ``include/mtp.h``); ``paper_2505_01059_gb300.mtp`` is its thin ctypes
binding.  Importing this package does not load the library; the binding loads
it on first use and raises if it is missing.
"""

__all__ = ["mtp", "workloads"]
