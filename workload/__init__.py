"""Seeded synthetic inputs for the punctured-eMBB receive path.

Input generation only (base matrices, transmit chain, slot grids, puncture
masks).  Both the CUDA path's tests and benchmark and the CPU oracle consume
these inputs; nothing here demaps, decodes or checks a CRC.
"""
from .basegraph import BaseGraph, make_base_graph, tree_base_graph, custom_base_graph  # noqa: F401
from .configs import (CB_DTYPE, TB_DTYPE, Workload, TBSpec, build, default_bgs,  # noqa: F401
                      tiny_fp32, large_fp32, mixed)
