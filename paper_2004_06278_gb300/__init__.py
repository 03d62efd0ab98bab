"""GB300 (sm_103a) implementation of the Squares counter-based RNG
(B. Widynski, arXiv:2004.06278).

The compute path is libsquares.so (hand-written CUDA behind the C ABI of
include/squares.h). ``_lib`` binds it entry point by entry point; the
helpers below only allocate torch tensors and pass their device pointers
and the current CUDA stream. Nothing here computes random numbers on the
host, and importing the package does not load the library: the first call
does, and it raises if the library was not built.
"""
from __future__ import annotations

from . import _lib
from ._lib import (  # noqa: F401  (re-exported C-ABI names)
    SQ_ECUDA, SQ_EINVAL, SQ_ERANGE, SQ_KERNEL_BATCH, SQ_KERNEL_FUSED, SQ_KERNEL_NORMAL_F32,
    SQ_KERNEL_U32, SQ_KERNEL_U64, SQ_KERNEL_UNIFORM2_F32, SQ_KERNEL_UNIFORM_BF16,
    SQ_KERNEL_UNIFORM_F32, SQ_KERNEL_UNIFORM_F64, SQ_NUM_KERNELS, SQ_OK, SquaresError, load,
    sq_abi_version, sq_autotune, sq_build_id, sq_autotune_batch, sq_autotune_load, sq_autotune_save, sq_batch,
    sq_batch_graph_create, sq_batch_validate, sq_debug_fail_next, sq_fill_u32, sq_fused_stats, sq_get_config, sq_graph_destroy,
    sq_graph_launch, sq_keys_u32, sq_keys_u64, sq_last_error, sq_make_keys, sq_normal_f32,
    sq_num_variants, sq_set_config, sq_u32, sq_u32_strided, sq_u64, sq_u64_strided,
    sq_uniform2_f32, sq_uniform_bf16, sq_uniform_f32, sq_uniform_f64, sq_variant_name)

__all__ = [n for n in dir(_lib) if n.startswith(("sq_", "SQ_"))] + [
    "SquaresError", "load", "make_keys", "u32", "u64", "uniform_f32", "uniform_bf16",
    "normal_f32", "uniform2_f32", "uniform_f64", "u32_strided", "u64_strided", "keys_u32",
    "keys_u64", "batch", "fused_stats"]


def _stream(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def make_keys(seed: int, n: int):
    """n "different digits" keys (Section 3) as a numpy uint64 array."""
    import numpy as np

    keys = np.empty(n, dtype=np.uint64)
    sq_make_keys(seed, n, keys.ctypes.data if n else 0)
    return keys


def _out(out, n, dtype, device):
    import torch

    if out is None:
        return torch.empty(n, dtype=dtype, device=device or "cuda")
    if not out.is_cuda or not out.is_contiguous() or out.numel() < n:
        raise ValueError("out must be a contiguous CUDA tensor with at least n elements")
    return out


def u32(key: int, ctr_base: int, n: int, out=None, stream=None, device=None):
    """squares32 at counters ctr_base .. ctr_base + n - 1 (torch.uint32)."""
    import torch

    out = _out(out, n, torch.uint32, device)
    sq_u32(key, ctr_base, n, out.data_ptr(), _stream(stream))
    return out


def u64(key: int, ctr_base: int, n: int, out=None, stream=None, device=None):
    """squares64 at counters ctr_base .. ctr_base + n - 1 (torch.uint64)."""
    import torch

    out = _out(out, n, torch.uint64, device)
    sq_u64(key, ctr_base, n, out.data_ptr(), _stream(stream))
    return out


def uniform_f32(key: int, ctr_base: int, n: int, out=None, stream=None, device=None):
    """Uniform float32 (squares32 >> 8) * 2^-24 in [0, 1), exact."""
    import torch

    out = _out(out, n, torch.float32, device)
    sq_uniform_f32(key, ctr_base, n, out.data_ptr(), _stream(stream))
    return out


def uniform_bf16(key: int, ctr_base: int, n: int, out=None, stream=None, device=None):
    """Uniform bfloat16 in [0, 1), rounded toward zero (torch.bfloat16)."""
    import torch

    out = _out(out, n, torch.bfloat16, device)
    sq_uniform_bf16(key, ctr_base, n, out.data_ptr(), _stream(stream))
    return out


def normal_f32(key: int, ctr_base: int, n: int, out=None, stream=None, device=None):
    """Box-Muller normals (torch.float32); squares64(ctr_base + j) gives outputs
    2j and 2j + 1."""
    import torch

    out = _out(out, n, torch.float32, device)
    sq_normal_f32(key, ctr_base, n, out.data_ptr(), _stream(stream))
    return out


def uniform2_f32(key: int, ctr_base: int, n: int, out=None, stream=None, device=None):
    """Two float uniforms per squares64 output (upper half, then lower)."""
    import torch

    out = _out(out, n, torch.float32, device)
    sq_uniform2_f32(key, ctr_base, n, out.data_ptr(), _stream(stream))
    return out


def uniform_f64(key: int, ctr_base: int, n: int, out=None, stream=None, device=None):
    """53-bit double uniforms from squares64 (torch.float64)."""
    import torch

    out = _out(out, n, torch.float64, device)
    sq_uniform_f64(key, ctr_base, n, out.data_ptr(), _stream(stream))
    return out


def u32_strided(key: int, ctr_base: int, stride: int, n: int, out=None, stream=None, device=None):
    """squares32 at counters ctr_base + i*stride (torch.uint32)."""
    import torch

    out = _out(out, n, torch.uint32, device)
    sq_u32_strided(key, ctr_base, stride, n, out.data_ptr(), _stream(stream))
    return out


def u64_strided(key: int, ctr_base: int, stride: int, n: int, out=None, stream=None, device=None):
    """squares64 at counters ctr_base + i*stride (torch.uint64)."""
    import torch

    out = _out(out, n, torch.uint64, device)
    sq_u64_strided(key, ctr_base, stride, n, out.data_ptr(), _stream(stream))
    return out


def keys_u32(keys, ctr: int, out=None, stream=None):
    """squares32(ctr, keys[i]) for a CUDA tensor of keys (key-counter mode)."""
    import torch

    out = _out(out, keys.numel(), torch.uint32, keys.device)
    sq_keys_u32(keys.data_ptr(), keys.numel(), ctr, out.data_ptr(), _stream(stream))
    return out


def keys_u64(keys, ctr: int, out=None, stream=None):
    """squares64(ctr, keys[i]) for a CUDA tensor of keys (key-counter mode)."""
    import torch

    out = _out(out, keys.numel(), torch.uint64, keys.device)
    sq_keys_u64(keys.data_ptr(), keys.numel(), ctr, out.data_ptr(), _stream(stream))
    return out


def batch(keys, ctr_bases, lengths, offsets, out, stream=None):
    """Ragged batch into `out` (torch.uint32); all inputs are CUDA tensors."""
    sq_batch(keys.data_ptr(), ctr_bases.data_ptr(), lengths.data_ptr(), offsets.data_ptr(),
             keys.numel(), out.data_ptr(), _stream(stream))
    return out


def fused_stats(keys, ctr_bases, ctrs_per_stream: int, stream=None):
    """(xor uint32[S], sum_top uint64[S], hist uint64[256]) on the device."""
    import torch

    S = keys.numel()
    xor = torch.empty(S, dtype=torch.uint32, device=keys.device)
    sums = torch.empty(S, dtype=torch.uint64, device=keys.device)
    hist = torch.empty(256, dtype=torch.uint64, device=keys.device)
    sq_fused_stats(keys.data_ptr(), ctr_bases.data_ptr(), S, ctrs_per_stream, xor.data_ptr(),
                   sums.data_ptr(), hist.data_ptr(), _stream(stream))
    return xor, sums, hist
