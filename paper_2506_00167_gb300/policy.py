"""Puncturing allocations on the device: the RP and SeF policies, the feasibility enforcer, SC masks,
and the RT O-DU codebook (policy forward pass + enforcer).

Thin wrappers over ``ldpc_puncture_alloc``, ``ldpc_feasibility_enforce``,
``ldpc_sc_mask`` and ``ldpc_rt_odu_codebook`` (see ``include/ldpcgb.h``):
they check shapes and dtypes,
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


def rt_odu_codebook(alloc: torch.Tensor, w1: torch.Tensor, b1: torch.Tensor, w2: torch.Tensor, b2: torch.Tensor,
                    noise: torch.Tensor, L: int):
    """alloc int32 [T, E]; weights float32 w1 [H, E+1], b1 [H], w2 [2E, H], b2 [2E]; noise float32 [T, J, E]
    -> (codebook int32 [T, J, E], actions float32 [T, J, E], status int32 [T, J])."""
    T, E = alloc.shape
    H = w1.shape[0]
    J = noise.shape[1]
    _need(alloc, torch.int32, (T, E), "alloc")
    _need(w1, torch.float32, (H, E + 1), "w1")
    _need(b1, torch.float32, (H,), "b1")
    _need(w2, torch.float32, (2 * E, H), "w2")
    _need(b2, torch.float32, (2 * E,), "b2")
    _need(noise, torch.float32, (T, J, E), "noise")
    book = torch.empty((T, J, E), dtype=torch.int32, device=alloc.device)
    act = torch.empty((T, J, E), dtype=torch.float32, device=alloc.device)
    status = torch.empty((T, J), dtype=torch.int32, device=alloc.device)
    abi.check(abi.load().ldpc_rt_odu_codebook(T, E, H, J, int(L), _ptr(alloc), _ptr(w1), _ptr(b1), _ptr(w2),
                                              _ptr(b2), _ptr(noise), _ptr(book), _ptr(act), _ptr(status),
                                              _stream()), "ldpc_rt_odu_codebook")
    return book, act, status
