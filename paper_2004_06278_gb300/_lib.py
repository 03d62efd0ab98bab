"""ctypes binding of libsquares.so (include/squares.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name, converts a non-zero status into ``SquaresError`` and
returns nothing else. Pointers are plain integers (``tensor.data_ptr()``),
streams are ``cudaStream_t`` handles as integers (0 = legacy default
stream). The library must have been built (``build.build()``); loading never
falls back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsquares.so")

SQ_OK = 0
SQ_EINVAL = -1
SQ_ECUDA = -2
SQ_ERANGE = -3

SQ_KERNEL_U32 = 0
SQ_KERNEL_U64 = 1
SQ_KERNEL_BATCH = 2
SQ_KERNEL_UNIFORM_F32 = 3
SQ_KERNEL_UNIFORM_BF16 = 4
SQ_KERNEL_NORMAL_F32 = 5
SQ_KERNEL_FUSED = 6
SQ_KERNEL_UNIFORM2_F32 = 7
SQ_KERNEL_UNIFORM_F64 = 8
SQ_NUM_KERNELS = 9

_STATUS = {SQ_EINVAL: "SQ_EINVAL", SQ_ECUDA: "SQ_ECUDA", SQ_ERANGE: "SQ_ERANGE"}


class SquaresError(RuntimeError):
    def __init__(self, fn: str, status: int, message: str):
        super().__init__(f"{fn}: {_STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class sq_launch_config(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("block", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_u64 = ctypes.c_uint64
_sz = ctypes.c_size_t
_p = ctypes.c_void_p
_i = ctypes.c_int

# name -> argument types; every entry point returns int status unless noted.
_SIGNATURES = {
    "sq_make_keys": [_u64, _sz, _p],
    "sq_debug_fail_next": [ctypes.c_char_p],
    "sq_u32": [_u64, _u64, _sz, _p, _p],
    "sq_u64": [_u64, _u64, _sz, _p, _p],
    "sq_u32_strided": [_u64, _u64, _u64, _sz, _p, _p],
    "sq_u64_strided": [_u64, _u64, _u64, _sz, _p, _p],
    "sq_keys_u32": [_p, _sz, _u64, _p, _p],
    "sq_keys_u64": [_p, _sz, _u64, _p, _p],
    "sq_uniform2_f32": [_u64, _u64, _sz, _p, _p],
    "sq_uniform_f64": [_u64, _u64, _sz, _p, _p],
    "sq_fill_u32": [ctypes.c_uint32, _sz, _p, ctypes.POINTER(sq_launch_config), ctypes.c_uint32, _p],
    "sq_batch": [_p, _p, _p, _p, _sz, _p, _p],
    "sq_batch_validate": [_p, _p, _sz, _p],
    "sq_uniform_f32": [_u64, _u64, _sz, _p, _p],
    "sq_uniform_bf16": [_u64, _u64, _sz, _p, _p],
    "sq_normal_f32": [_u64, _u64, _sz, _p, _p],
    "sq_fused_stats": [_p, _p, _sz, _u64, _p, _p, _p, _p],
    "sq_num_variants": [_i],
    "sq_get_config": [_i, _sz, ctypes.POINTER(sq_launch_config)],
    "sq_set_config": [_i, _sz, ctypes.POINTER(sq_launch_config)],
    "sq_autotune": [_i, _sz],
    "sq_autotune_batch": [_p, _p, _p, _p, _sz, _p],
    "sq_autotune_save": [ctypes.c_char_p],
    "sq_autotune_load": [ctypes.c_char_p],
    "sq_batch_graph_create": [_p, _p, _p, _p, _sz, _p, ctypes.POINTER(_p)],
    "sq_graph_launch": [_p, _p],
    "sq_graph_destroy": [_p],
}
_OTHER = {
    "sq_last_error": (ctypes.c_char_p, []),
    "sq_abi_version": (_i, []),
    "sq_build_id": (ctypes.c_char_p, []),
    "sq_variant_name": (ctypes.c_char_p, [_i, _i]),
}

_lib = None
_lock = threading.Lock()


def load() -> ctypes.CDLL:
    """Load libsquares.so; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = _i
        for name, (res, args) in _OTHER.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def declared_symbols() -> list[str]:
    return sorted(list(_SIGNATURES) + list(_OTHER))


def _check(fn: str, status: int) -> None:
    if status != SQ_OK:
        msg = load().sq_last_error()
        raise SquaresError(fn, status, msg.decode() if msg else "")


def _call(name: str, *args) -> None:
    _check(name, getattr(load(), name)(*args))


def sq_last_error() -> str:
    return load().sq_last_error().decode()


def sq_abi_version() -> int:
    return int(load().sq_abi_version())


def sq_build_id() -> str:
    return load().sq_build_id().decode()


def sq_debug_fail_next(entry_point: str | None) -> None:
    _call("sq_debug_fail_next", entry_point.encode() if entry_point else None)


def sq_make_keys(seed: int, n: int, keys_ptr: int) -> None:
    _call("sq_make_keys", seed, n, keys_ptr)


def sq_u32(key: int, ctr_base: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _call("sq_u32", key, ctr_base, n, out_ptr, stream)


def sq_u64(key: int, ctr_base: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _call("sq_u64", key, ctr_base, n, out_ptr, stream)


def sq_u32_strided(key: int, ctr_base: int, stride: int, n: int, out_ptr: int,
                   stream: int = 0) -> None:
    _call("sq_u32_strided", key, ctr_base, stride, n, out_ptr, stream)


def sq_u64_strided(key: int, ctr_base: int, stride: int, n: int, out_ptr: int,
                   stream: int = 0) -> None:
    _call("sq_u64_strided", key, ctr_base, stride, n, out_ptr, stream)


def sq_keys_u32(keys_ptr: int, nkeys: int, ctr: int, out_ptr: int, stream: int = 0) -> None:
    _call("sq_keys_u32", keys_ptr, nkeys, ctr, out_ptr, stream)


def sq_keys_u64(keys_ptr: int, nkeys: int, ctr: int, out_ptr: int, stream: int = 0) -> None:
    _call("sq_keys_u64", keys_ptr, nkeys, ctr, out_ptr, stream)


def sq_uniform2_f32(key: int, ctr_base: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _call("sq_uniform2_f32", key, ctr_base, n, out_ptr, stream)


def sq_uniform_f64(key: int, ctr_base: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _call("sq_uniform_f64", key, ctr_base, n, out_ptr, stream)


def sq_fill_u32(value: int, n: int, out_ptr: int, config: tuple | None = None,
                pause_ns: int = 0, stream: int = 0) -> None:
    """config: (variant, block, ctas_per_sm) as for SQ_KERNEL_U32, or None."""
    cfg = None if config is None else ctypes.byref(sq_launch_config(*config, 0))
    _call("sq_fill_u32", value, n, out_ptr, cfg, pause_ns, stream)


def sq_batch(keys_ptr: int, bases_ptr: int, lengths_ptr: int, offsets_ptr: int, nstreams: int,
             out_ptr: int, stream: int = 0) -> None:
    _call("sq_batch", keys_ptr, bases_ptr, lengths_ptr, offsets_ptr, nstreams, out_ptr, stream)


def sq_batch_validate(lengths_ptr: int, offsets_ptr: int, nstreams: int, stream: int = 0) -> None:
    _call("sq_batch_validate", lengths_ptr, offsets_ptr, nstreams, stream)


def sq_uniform_f32(key: int, ctr_base: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _call("sq_uniform_f32", key, ctr_base, n, out_ptr, stream)


def sq_uniform_bf16(key: int, ctr_base: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _call("sq_uniform_bf16", key, ctr_base, n, out_ptr, stream)


def sq_normal_f32(key: int, ctr_base: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _call("sq_normal_f32", key, ctr_base, n, out_ptr, stream)


def sq_fused_stats(keys_ptr: int, bases_ptr: int, nstreams: int, ctrs_per_stream: int,
                   xor_ptr: int, sum_ptr: int, hist_ptr: int, stream: int = 0) -> None:
    _call("sq_fused_stats", keys_ptr, bases_ptr, nstreams, ctrs_per_stream, xor_ptr, sum_ptr,
          hist_ptr, stream)


def sq_num_variants(kernel_id: int) -> int:
    r = int(load().sq_num_variants(kernel_id))
    if r < 0:
        _check("sq_num_variants", r)
    return r


def sq_variant_name(kernel_id: int, variant: int) -> str | None:
    r = load().sq_variant_name(kernel_id, variant)
    return r.decode() if r else None


def sq_get_config(kernel_id: int, n: int) -> sq_launch_config:
    cfg = sq_launch_config()
    _call("sq_get_config", kernel_id, n, ctypes.byref(cfg))
    return cfg


def sq_set_config(kernel_id: int, n: int, variant: int, block: int, ctas_per_sm: int) -> None:
    cfg = sq_launch_config(variant, block, ctas_per_sm, 0)
    _call("sq_set_config", kernel_id, n, ctypes.byref(cfg))


def sq_autotune(kernel_id: int, n_hint: int) -> None:
    _call("sq_autotune", kernel_id, n_hint)


def sq_autotune_batch(keys_ptr: int, bases_ptr: int, lengths_ptr: int, offsets_ptr: int,
                      nstreams: int, out_ptr: int) -> None:
    _call("sq_autotune_batch", keys_ptr, bases_ptr, lengths_ptr, offsets_ptr, nstreams, out_ptr)


def sq_autotune_save(path: str) -> None:
    _call("sq_autotune_save", path.encode())


def sq_autotune_load(path: str) -> None:
    _call("sq_autotune_load", path.encode())


def sq_batch_graph_create(keys_ptr: int, bases_ptr: int, lengths_ptr: int, offsets_ptr: int,
                          nstreams: int, out_ptr: int) -> int:
    g = _p()
    _call("sq_batch_graph_create", keys_ptr, bases_ptr, lengths_ptr, offsets_ptr, nstreams,
          out_ptr, ctypes.byref(g))
    return int(g.value or 0)


def sq_graph_launch(graph: int, stream: int = 0) -> None:
    _call("sq_graph_launch", graph, stream)


def sq_graph_destroy(graph: int) -> None:
    _call("sq_graph_destroy", graph)
