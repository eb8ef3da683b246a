"""Puncturing allocations on the device: the RP and SeF policies, the feasibility enforcer, SC masks.

Thin wrappers over ``ldpc_puncture_alloc``, ``ldpc_feasibility_enforce`` and
``ldpc_sc_mask`` (see ``include/ldpcgb.h``): they check shapes and dtypes,
allocate the outputs as torch tensors on the inputs' device and enqueue on the
current stream.  Every step runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import abi

N_MINISLOT = 7
SYM_PER_SLOT = 14


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype, shape, name: str) -> None:
    if not t.is_cuda or t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor of shape {tuple(shape)}")


def puncture_alloc(alloc: torch.Tensor, demand: torch.Tensor, policy: str):
    """alloc int32 [T, E], demand int32 [T, 7] -> (punct int32 [T, 7, E], status int32 [T, 7])."""
    T, E = alloc.shape
    _need(alloc, torch.int32, (T, E), "alloc")
    _need(demand, torch.int32, (T, N_MINISLOT), "demand")
    code = {"rp": abi.POLICY_RP, "sef": abi.POLICY_SEF}[policy]
    punct = torch.empty((T, N_MINISLOT, E), dtype=torch.int32, device=alloc.device)
    status = torch.empty((T, N_MINISLOT), dtype=torch.int32, device=alloc.device)
    abi.check(abi.load().ldpc_puncture_alloc(code, T, E, _ptr(alloc), _ptr(demand), _ptr(punct), _ptr(status),
                                             _stream()), "ldpc_puncture_alloc")
    return punct, status


def enforce(punct_real: torch.Tensor, alloc: torch.Tensor, total: torch.Tensor):
    """punct_real float32 [P, E], alloc int32 [P, E], total int32 [P] -> (punct int32 [P, E], status int32 [P])."""
    P, E = punct_real.shape
    _need(punct_real, torch.float32, (P, E), "punct_real")
    _need(alloc, torch.int32, (P, E), "alloc")
    _need(total, torch.int32, (P,), "total")
    punct = torch.empty((P, E), dtype=torch.int32, device=alloc.device)
    status = torch.empty((P,), dtype=torch.int32, device=alloc.device)
    abi.check(abi.load().ldpc_feasibility_enforce(P, E, _ptr(punct_real), _ptr(alloc), _ptr(total), _ptr(punct),
                                                  _ptr(status), _stream()), "ldpc_feasibility_enforce")
    return punct, status


def sc_mask(alloc: torch.Tensor, punct: torch.Tensor, words_per_symbol: int | None = None) -> torch.Tensor:
    """alloc int32 [T, E], punct int32 [T, 7, E] -> uint32 bitmap as int32 [T, 14, words] (bit b of word w: SC 32w+b)."""
    T, E = alloc.shape
    _need(alloc, torch.int32, (T, E), "alloc")
    _need(punct, torch.int32, (T, N_MINISLOT, E), "punct")
    if words_per_symbol is None:
        words_per_symbol = max(1, (int(alloc.sum(dim=1).max().item()) + 31) // 32) if T else 1
    mask = torch.empty((T, SYM_PER_SLOT, words_per_symbol), dtype=torch.int32, device=alloc.device)
    abi.check(abi.load().ldpc_sc_mask(T, E, _ptr(alloc), _ptr(punct), int(words_per_symbol), _ptr(mask),
                                      _stream()), "ldpc_sc_mask")
    return mask
