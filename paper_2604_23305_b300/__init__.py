"""B300-native (sm_103a) hot path of the gateau submillimetre TOD simulator (arXiv 2604.23305).

The compute path lives in libgateau_b300.so (CUDA kernels behind the C ABI of
include/gateau.h).  Importing this package loads nothing; ``Plan`` loads the
library on first use and raises if it has not been built.
"""
from .plan import Plan, hex_offsets, run_batch  # noqa: F401

__all__ = ["Plan", "hex_offsets", "run_batch"]
