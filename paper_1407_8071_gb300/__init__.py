"""GB300-native ensemble of independent bootstrap particle filters (arXiv:1407.8071).

The hot path -- Euler-Maruyama propagation, Gaussian log-weights, per-filter
FP64 normalisation, systematic resampling with a gather, and the average over
the M filters -- runs in the sm_103a kernels of libpf_gb300.so behind the C
ABI of include/pf.h; ``paper_1407_8071_gb300.pf`` is its ctypes binding.
"""
from . import workloads  # noqa: F401
