"""Level-wise wavelet tree on one GB300 (sm_103a).

GPU construction and batched access/rank/select of the extended level-wise
wavelet tree of "GPU Implementation of the Wavelet Tree" (arXiv 2505.03372),
behind the C ABI of ``libwt.so`` (include/wt.h).  This package holds the CUDA
sources (``csrc/``), their in-tree build (``_build.py``), the ctypes binding
(``binding.py``) and the seeded workload generators (``workloads.py``).
"""
from .binding import (  # noqa: F401
    EXPORT_BITS, EXPORT_C, EXPORT_CODES, EXPORT_L1, EXPORT_L2, EXPORT_LENS, EXPORT_NODES, EXPORT_S0, EXPORT_S1,
    WT_EINVAL, WT_EQUERY, WT_ESYMBOL, WT_ETIMEOUT, WT_OK, Batch, Tree, WTError, build, profile_enable, profile_launches,
    profile_report, profile_reset, status_str,
)
