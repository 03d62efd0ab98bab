"""CPU oracle for the Squares counter-based generator (arXiv:2004.06278).

TEST INFRASTRUCTURE ONLY. Nothing in the product package imports this module;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may. It wraps ``squares_oracle.c`` (plain C, compiled with gcc)
through ctypes and adds nothing to its arithmetic: the Python side only
allocates numpy arrays, splits large fills into counter ranges that worker
threads evaluate (ctypes releases the GIL during the call), and builds the
shared object.

Every function names the paper passage it follows:
  squares32 / fill32 / pairs32 ... Section 2 (four-round generator)
  squares64 / fill64 / pairs64 ... Section 5 (five-round, 64-bit output)
  batch32 ........................ ragged batch of Section 2 streams
  fill32_strided / fill64_strided  strided counters (Section 4)
  uniform_f32 / uniform_bf16 ..... float conversion (Section 5 prose), FP64
  uniform2_f32 / uniform_f64 ..... two floats / one 53-bit double per squares64
  uniform53_of ................... that double for given 64-bit values
  normal_f64 ..................... Box-Muller on squares64 halves, FP64
  box_muller_f64 ................. the same pair for given 32-bit halves
  fused_stats .................... XOR / top-byte sum / top-byte histogram
  make_keys ...................... "different digits" keys (Section 3)
  squares_w / hist_w ............. reduced-width analogue for brute force
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "squares_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_squares.so")
_lock = threading.Lock()
_lib = None

_u64 = ctypes.c_uint64
_i = ctypes.c_int
_u = ctypes.c_uint
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC", _SRC,
             "-o", tmp, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        sigs = {
            "oracle_squares32": (ctypes.c_uint32, [_u64, _u64]),
            "oracle_squares64": (_u64, [_u64, _u64]),
            "oracle_squares_w": (_u64, [_u64, _u64, _u, _u, _i, _i]),
            "oracle_hist_w": (None, [_u64, _u, _u, _i, _p]),
            "oracle_hist_w_range": (None, [_u64, _u, _u, _i, _u64, _u64, _p]),
            "oracle_fill32": (None, [_u64, _u64, _u64, _p]),
            "oracle_fill64": (None, [_u64, _u64, _u64, _p]),
            "oracle_fill32_strided": (None, [_u64, _u64, _u64, _u64, _p]),
            "oracle_fill64_strided": (None, [_u64, _u64, _u64, _u64, _p]),
            "oracle_uniform2_f32": (None, [_u64, _u64, _u64, _p]),
            "oracle_uniform_f64": (None, [_u64, _u64, _u64, _p]),
            "oracle_pairs32": (None, [_p, _p, _u64, _p]),
            "oracle_pairs64": (None, [_p, _p, _u64, _p]),
            "oracle_batch32": (None, [_p, _p, _p, _p, _u64, _p]),
            "oracle_uniform_f32": (None, [_u64, _u64, _u64, _p]),
            "oracle_uniform_bf16": (None, [_u64, _u64, _u64, _p]),
            "oracle_normal_f64": (None, [_u64, _u64, _u64, _p]),
            "oracle_box_muller_f64": (None, [_p, _p, _u64, _p]),
            "oracle_uniform53_of": (None, [_p, _u64, _p]),
            "oracle_fused_stats": (None, [_p, _p, _u64, _u64, _p, _p, _p]),
            "oracle_make_keys": (_i, [_u64, _u64, _p]),
            "oracle_splitmix64": (None, [_u64, _u64, _p]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _chunks(n: int, threads: int, min_chunk: int = 1 << 16):
    """Split [0, n) into at most `threads` contiguous ranges."""
    if n <= 0:
        return []
    parts = max(1, min(threads, (n + min_chunk - 1) // min_chunk))
    step = (n + parts - 1) // parts
    return [(a, min(n, a + step)) for a in range(0, n, step)]


def _parallel(fn, ranges, threads):
    if len(ranges) <= 1:
        for a, b in ranges:
            fn(a, b)
        return
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda r: fn(*r), ranges))


M64 = (1 << 64) - 1


# --- generator, Section 2 and Section 5 -----------------------------------

def squares32(ctr: int, key: int) -> int:
    """squares32(ctr, key), Section 2."""
    return int(_load().oracle_squares32(ctr & M64, key & M64))


def squares64(ctr: int, key: int) -> int:
    """squares64(ctr, key), Section 5."""
    return int(_load().oracle_squares64(ctr & M64, key & M64))


def squares_w(ctr: int, key: int, w: int, rounds: int, use_z: bool = True,
              wide: bool = False) -> int:
    """Reduced-width analogue (w-bit state, rotation by w/2)."""
    return int(_load().oracle_squares_w(ctr, key, w, rounds, int(use_z), int(wide)))


def hist_w(key: int, w: int, rounds: int = 4, use_z: bool = True,
           threads: int | None = None) -> np.ndarray:
    """Histogram of the narrow reduced-width output over all 2^w counters
    (counter ranges on worker threads, one histogram each, summed)."""
    lib = _load()
    threads = threads or default_threads()
    ranges = _chunks(1 << w, threads, min_chunk=1 << 22)
    hs = [np.zeros(1 << (w // 2), dtype=np.uint64) for _ in ranges]

    def run(i):
        a, b = ranges[i]
        lib.oracle_hist_w_range(key, w, rounds, int(use_z), a, b, _ptr(hs[i]))

    if len(ranges) <= 1:
        for i in range(len(ranges)):
            run(i)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(run, range(len(ranges))))
    return np.sum(hs, axis=0, dtype=np.uint64)


def fill32(key: int, base: int, n: int, threads: int | None = None) -> np.ndarray:
    """out[i] = squares32(base + i mod 2^64, key)."""
    lib = _load()
    out = np.empty(n, dtype=np.uint32)
    threads = threads or default_threads()
    addr = out.ctypes.data

    def run(a, b):
        lib.oracle_fill32(key, (base + a) & M64, b - a, addr + 4 * a)

    _parallel(run, _chunks(n, threads), threads)
    return out


def fill64(key: int, base: int, n: int, threads: int | None = None) -> np.ndarray:
    """out[i] = squares64(base + i mod 2^64, key)."""
    lib = _load()
    out = np.empty(n, dtype=np.uint64)
    threads = threads or default_threads()
    addr = out.ctypes.data

    def run(a, b):
        lib.oracle_fill64(key, (base + a) & M64, b - a, addr + 8 * a)

    _parallel(run, _chunks(n, threads), threads)
    return out


def fill32_strided(key: int, base: int, stride: int, n: int) -> np.ndarray:
    """out[i] = squares32(base + i*stride mod 2^64, key) (Section 4)."""
    out = np.empty(n, dtype=np.uint32)
    _load().oracle_fill32_strided(key, base & M64, stride & M64, n, out.ctypes.data)
    return out


def fill64_strided(key: int, base: int, stride: int, n: int) -> np.ndarray:
    """out[i] = squares64(base + i*stride mod 2^64, key) (Section 4)."""
    out = np.empty(n, dtype=np.uint64)
    _load().oracle_fill64_strided(key, base & M64, stride & M64, n, out.ctypes.data)
    return out


def pairs32(ctrs: np.ndarray, keys: np.ndarray) -> np.ndarray:
    """out[i] = squares32(ctrs[i], keys[i])."""
    ctrs = np.ascontiguousarray(ctrs, dtype=np.uint64)
    keys = np.ascontiguousarray(np.broadcast_to(keys, ctrs.shape), dtype=np.uint64)
    out = np.empty(ctrs.shape, dtype=np.uint32)
    _load().oracle_pairs32(_ptr(ctrs), _ptr(keys), ctrs.size, _ptr(out))
    return out


def pairs64(ctrs: np.ndarray, keys: np.ndarray) -> np.ndarray:
    """out[i] = squares64(ctrs[i], keys[i])."""
    ctrs = np.ascontiguousarray(ctrs, dtype=np.uint64)
    keys = np.ascontiguousarray(np.broadcast_to(keys, ctrs.shape), dtype=np.uint64)
    out = np.empty(ctrs.shape, dtype=np.uint64)
    _load().oracle_pairs64(_ptr(ctrs), _ptr(keys), ctrs.size, _ptr(out))
    return out


def batch32(keys, bases, lengths, offsets, out: np.ndarray) -> np.ndarray:
    """Ragged batch: out[offsets[s] + i] = squares32(bases[s] + i, keys[s])."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    bases = np.ascontiguousarray(bases, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    assert out.dtype == np.uint32
    _load().oracle_batch32(_ptr(keys), _ptr(bases), _ptr(lengths), _ptr(offsets),
                           keys.size, _ptr(out))
    return out


# --- distribution transforms, FP64 ----------------------------------------

def uniform_f32(key: int, base: int, n: int, threads: int | None = None) -> np.ndarray:
    """Uniform [0,1): floor(squares32 / 2^8) / 2^24."""
    lib = _load()
    out = np.empty(n, dtype=np.float32)
    threads = threads or default_threads()
    addr = out.ctypes.data
    _parallel(lambda a, b: lib.oracle_uniform_f32(key, (base + a) & M64, b - a, addr + 4 * a),
              _chunks(n, threads), threads)
    return out


def uniform_bf16(key: int, base: int, n: int, threads: int | None = None) -> np.ndarray:
    """The uniform above rounded toward zero to bfloat16; returns the bits."""
    lib = _load()
    out = np.empty(n, dtype=np.uint16)
    threads = threads or default_threads()
    addr = out.ctypes.data
    _parallel(lambda a, b: lib.oracle_uniform_bf16(key, (base + a) & M64, b - a, addr + 2 * a),
              _chunks(n, threads), threads)
    return out


def uniform2_f32(key: int, base: int, n: int) -> np.ndarray:
    """Two float uniforms per squares64 output: upper half, then lower."""
    out = np.empty(n, dtype=np.float32)
    _load().oracle_uniform2_f32(key, base & M64, n, out.ctypes.data)
    return out


def uniform_f64(key: int, base: int, n: int) -> np.ndarray:
    """53-bit double uniforms floor(squares64 / 2^11) / 2^53."""
    out = np.empty(n, dtype=np.float64)
    _load().oracle_uniform_f64(key, base & M64, n, out.ctypes.data)
    return out


def normal_f64(key: int, base: int, n: int, threads: int | None = None) -> np.ndarray:
    """Box-Muller normals in FP64; squares64(base + j) feeds outputs 2j, 2j+1."""
    lib = _load()
    out = np.empty(n, dtype=np.float64)
    threads = threads or default_threads()
    addr = out.ctypes.data
    npairs = (n + 1) // 2

    def run(a, b):  # a, b index pairs
        count = min(n, 2 * b) - 2 * a
        lib.oracle_normal_f64(key, (base + a) & M64, count, addr + 8 * 2 * a)

    _parallel(run, _chunks(npairs, threads), threads)
    return out


def uniform53_of(v) -> np.ndarray:
    """floor(v / 2^11) / 2^53 as doubles, for given 64-bit values."""
    v = np.ascontiguousarray(v, dtype=np.uint64)
    out = np.empty(v.shape, dtype=np.float64)
    _load().oracle_uniform53_of(_ptr(v), v.size, _ptr(out))
    return out


def box_muller_f64(hi, lo, threads: int | None = None) -> np.ndarray:
    """Box-Muller pairs in FP64 for given upper / lower halves: row i is
    (r cos theta, r sin theta) with u1 = (hi[i] + 1) / 2^32 and
    theta = 2 pi lo[i] / 2^32."""
    lib = _load()
    hi = np.ascontiguousarray(hi, dtype=np.uint32)
    lo = np.ascontiguousarray(lo, dtype=np.uint32)
    assert hi.shape == lo.shape and hi.ndim == 1
    out = np.empty((hi.size, 2), dtype=np.float64)
    threads = threads or default_threads()

    def run(a, b):
        lib.oracle_box_muller_f64(_ptr(hi) + 4 * a, _ptr(lo) + 4 * a, b - a, _ptr(out) + 16 * a)

    _parallel(run, _chunks(hi.size, threads), threads)
    return out


# --- generation-only statistics -------------------------------------------

def fused_stats(keys, bases, ctrs_per_stream: int, threads: int | None = None):
    """Per-stream XOR and top-byte sum, and the global top-byte histogram."""
    lib = _load()
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    bases = np.ascontiguousarray(bases, dtype=np.uint64)
    S = keys.size
    xor_out = np.empty(S, dtype=np.uint32)
    sum_out = np.empty(S, dtype=np.uint64)
    threads = threads or default_threads()
    ranges = _chunks(S, threads, min_chunk=1)
    hists = [np.zeros(256, dtype=np.uint64) for _ in ranges]

    def run(idx):
        a, b = ranges[idx]
        lib.oracle_fused_stats(keys.ctypes.data + 8 * a, bases.ctypes.data + 8 * a,
                               b - a, ctrs_per_stream, xor_out.ctypes.data + 4 * a,
                               sum_out.ctypes.data + 8 * a, _ptr(hists[idx]))

    if len(ranges) <= 1:
        for i in range(len(ranges)):
            run(i)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(run, range(len(ranges))))
    hist = np.zeros(256, dtype=np.uint64)
    for h in hists:
        hist += h
    return xor_out, sum_out, hist


# --- keys, Section 3 --------------------------------------------------------

def make_keys(seed: int, n: int) -> np.ndarray:
    """n distinct "different digits" keys, deterministic in the seed."""
    out = np.empty(n, dtype=np.uint64)
    rc = _load().oracle_make_keys(seed & M64, n, _ptr(out) if n else 0)
    if rc != 0:
        raise MemoryError("oracle_make_keys could not allocate its table")
    return out


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The digit source of make_keys (Steele, Lea, Flood 2014)."""
    out = np.empty(n, dtype=np.uint64)
    _load().oracle_splitmix64(seed & M64, n, _ptr(out) if n else 0)
    return out
