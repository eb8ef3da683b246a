"""GB300 (sm_103a) receive path for URLLC-punctured eMBB transport blocks.

puncture flushing + max-log demap -> layered offset-min-sum QC-LDPC decode ->
TB CRC-24 -> goodput (eq. 1) and reward (eq. 2), as hand-written CUDA kernels
behind the C-ABI in ``include/ldpcgb.h`` (``libldpcgb.so``).  This package is
the ctypes binding; it needs the built library and a CUDA device.
"""
from .abi import LdpcError, load, CB_NP, TB_NP, MODES  # noqa: F401
from .session import Session, Batch, Graph, Server  # noqa: F401

__all__ = ["Session", "Batch", "Graph", "Server", "LdpcError", "load", "CB_NP", "TB_NP", "MODES"]
