"""GB300 (sm_103a) PAC stochastic aggregation: the hot path of SIMD-PAC-DB
(arXiv 2603.15023) as hand-written CUDA behind a C ABI (``include/pac.h``).

``binding`` is the ctypes layer with the C entry-point names; ``inputs``
draws seeded synthetic columns shaped like the paper's workloads.
"""
from . import binding  # noqa: F401
