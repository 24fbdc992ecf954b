"""GB300-native molecular-dynamics hot path of the ms2 method (arXiv 1507.07548).

The compute runs in libms2.so (hand-written CUDA for sm_103a behind the C ABI in
include/ms2.h); `ms2` is its ctypes binding and `workloads` makes seeded
synthetic inputs.
"""
from . import workloads  # noqa: F401
