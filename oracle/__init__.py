"""FP64 CPU oracle for the Model Tensor Planning hot path (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the CUDA library: the C
source in ``mtp_oracle.c`` restates the paper's Alg. 1, Alg. 2, Defs. 1-3 and
Eqs. 2-7 in plain loops, and this module only marshals numpy arrays.
"""
from .oracle import *  # noqa: F401,F403
