"""The oracle against an independent 128-bit re-derivation of every round
(tests/int128_route.c: full 128-bit squares reduced modulo 2^64 by masking,
z = (ctr+1)*key as its own product, halves exchanged by shifting a doubled
128-bit value), on edge counters and keys and on random pairs. CPU only."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle
from tests import pins

M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def route(tmp_path_factory):
    import os

    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "int128_route.c")
    so = tmp_path_factory.mktemp("int128") / "libint128_route.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.r128_squares32.restype = ctypes.c_uint32
    lib.r128_squares32.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.r128_squares64.restype = ctypes.c_uint64
    lib.r128_squares64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    return lib


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    ctrs = [int(c) for c in rng.integers(0, 1 << 64, n, dtype=np.uint64)]
    keys = [int(k) for k in rng.integers(0, 1 << 64, n, dtype=np.uint64)]
    edge_keys = [0, 1, 2, M64, 1 << 63, (1 << 63) + 1, 0x5555555555555555] + \
        [int(k) for k in oracle.make_keys(3, 5)]
    for c in pins.EDGE_CTRS:
        for k in edge_keys:
            ctrs.append(c & M64)
            keys.append(k)
    return ctrs, keys


def test_squares32_matches_int128_route(route):
    ctrs, keys = _pairs(100_000, 1)
    got = oracle.pairs32(np.array(ctrs, dtype=np.uint64), np.array(keys, dtype=np.uint64))
    want = np.array([route.r128_squares32(c, k) for c, k in zip(ctrs, keys)], dtype=np.uint32)
    assert np.array_equal(got, want)


def test_squares64_matches_int128_route(route):
    ctrs, keys = _pairs(100_000, 2)
    got = oracle.pairs64(np.array(ctrs, dtype=np.uint64), np.array(keys, dtype=np.uint64))
    want = np.array([route.r128_squares64(c, k) for c, k in zip(ctrs, keys)], dtype=np.uint64)
    assert np.array_equal(got, want)


def test_int128_route_against_hand_worked_examples(route):
    """The route itself reproduces the hand-derived golden values."""
    pins.pin_hand_worked(lambda c, k: route.r128_squares32(c & M64, k & M64),
                         lambda c, k: route.r128_squares64(c & M64, k & M64))
