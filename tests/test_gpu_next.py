"""GPU parity of the entry points beyond the throughput path: strided
counters and key-counter mode (Section 4), two float uniforms per squares64
output and 53-bit double uniforms (Section 5), all bit for bit against the
oracle."""
import numpy as np
import pytest

import oracle
from paper_2004_06278_gb300 import _lib as C
from tests.gpu_util import Guarded, stream_handle, to_dev

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1


def _run(fn, elem, dtype, *args, n, off=0):
    g = Guarded(n * elem, off * elem)
    fn(*args, n, g.ptr, stream_handle())
    assert g.guards_intact()
    return g.payload(dtype)


@pytest.mark.parametrize("stride", [0, 1, 2, 3, 1 << 20, (1 << 63) + 1, M64])
def test_strided(gpu_lib, stride):
    key = int(gpu_lib.make_keys(21, 1)[0])
    base = M64 - 1000
    # around the vector paths' thresholds (1,024 squares32, 256 squares64
    # outputs) and ragged tails of their 16- and 4-value chunks
    for n in (1, 7, 255, 256, 1000, 1023, 1024, 1025, 4099, 300_001):
        for off in {n % 4, 3}:
            got32 = _run(C.sq_u32_strided, 4, np.uint32, key, base, stride, n=n, off=off)
            got64 = _run(C.sq_u64_strided, 8, np.uint64, key, base, stride, n=n, off=off % 2)
            assert np.array_equal(got32, oracle.fill32_strided(key, base, stride, n)), (stride, n, off)
            assert np.array_equal(got64, oracle.fill64_strided(key, base, stride, n)), (stride, n, off)


@pytest.mark.parametrize("ctr", [0, 1, 12345, M64])
def test_key_counter_mode(gpu_lib, ctr):
    """Section 4: the counter fixed (even at 0) and the keys varying."""
    keys = gpu_lib.make_keys(22, 100_003)
    d_keys = to_dev(keys)
    ctrs = np.full(keys.size, ctr, dtype=np.uint64)
    for fn, elem, dt, ref in ((C.sq_keys_u32, 4, np.uint32, oracle.pairs32),
                              (C.sq_keys_u64, 8, np.uint64, oracle.pairs64)):
        g = Guarded(keys.size * elem, elem)
        fn(d_keys.data_ptr(), keys.size, ctr, g.ptr, stream_handle())
        assert g.guards_intact()
        assert np.array_equal(g.payload(dt), ref(ctrs, keys))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 4097, 100_003])
def test_key_counter_mode_alignments(gpu_lib, n):
    """Both launch paths of key-counter mode: keys and output 16-byte
    aligned (four keys per thread per step for squares32, then the n mod 4
    tail; two for squares64, then an odd last key) and either misaligned
    (one key per thread)."""
    import torch

    keys = gpu_lib.make_keys(26, n + 1)
    ctr = 0xFEDCBA9876543210
    for koff in (0, 1):  # keys offset by one element: 8-byte aligned only
        d_keys = to_dev(keys)
        kptr = d_keys.data_ptr() + 8 * koff
        k = keys[koff:koff + n]
        ctrs = np.full(n, ctr, dtype=np.uint64)
        for fn, elem, dt, ref in ((C.sq_keys_u32, 4, np.uint32, oracle.pairs32),
                                  (C.sq_keys_u64, 8, np.uint64, oracle.pairs64)):
            for ooff in (0, elem):
                g = Guarded(n * elem, ooff)
                fn(kptr, n, ctr, g.ptr, stream_handle())
                assert g.guards_intact(), (koff, ooff)
                assert np.array_equal(g.payload(dt), ref(ctrs, k)), (koff, ooff)
        torch.cuda.synchronize()


@pytest.mark.parametrize("n", [1, 2, 3, 8, 9, 31, 1001, (1 << 20) + 5])
def test_uniform2_f32(gpu_lib, n):
    key = int(gpu_lib.make_keys(23, 1)[0])
    want = oracle.uniform2_f32(key, 77, n).view(np.uint32)
    for off in (0, 1, 2, 3):
        got = _run(C.sq_uniform2_f32, 4, np.float32, key, 77, n=n, off=off)
        assert np.array_equal(got.view(np.uint32), want), (n, off)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 1001, (1 << 20) + 3])
def test_uniform_f64(gpu_lib, n):
    key = int(gpu_lib.make_keys(24, 1)[0])
    base = M64 - 17
    want = oracle.uniform_f64(key, base, n).view(np.uint64)
    for off in (0, 1, 3):
        got = _run(C.sq_uniform_f64, 8, np.float64, key, base, n=n, off=off)
        assert np.array_equal(got.view(np.uint64), want), (n, off)


def test_uniform_f64_rare_values_inside_chunks(gpu_lib):
    """squares64 outputs below 2^43 (probability 2^-21 each) take the
    conversion's rare path, which the vector kernels run after the chunk
    when a lane flagged one: windows around such counters, found by
    scanning the oracle, in every launch variant and block size, at two
    output alignments, against the oracle."""
    key = int(gpu_lib.make_keys(24, 1)[0])
    v = oracle.fill64(key, 0, 1 << 24)
    rare = np.nonzero(v < np.uint64(1 << 43))[0]
    assert rare.size >= 2, rare.size
    kid = C.SQ_KERNEL_UNIFORM_F64
    try:
        for r in rare[:3]:
            base, n = int(r) - 3000, 6001
            want = oracle.uniform_f64(key, base, n).view(np.uint64)
            for variant in range(C.sq_num_variants(kid)):
                for block in (128, 256, 512):
                    C.sq_set_config(kid, 0, variant, block, 0)
                    for off in (0, 1):
                        got = _run(C.sq_uniform_f64, 8, np.float64, key, base, n=n, off=off)
                        assert np.array_equal(got.view(np.uint64), want), (int(r), variant, block, off)
    finally:
        C.sq_set_config(kid, 0, 0, 256, 0)


def test_uniform_f64_edge_integers(gpu_lib):
    """Outputs whose top bits are small exercise the exponent construction:
    found by scanning the oracle, then generated on the GPU one by one."""
    key = int(gpu_lib.make_keys(24, 1)[0])
    v = oracle.fill64(key, 0, 1 << 22)
    picks = np.argsort(v)[:50]
    for j in picks:
        got = _run(C.sq_uniform_f64, 8, np.float64, key, int(j), n=1)
        assert got.view(np.uint64)[0] == oracle.uniform_f64(key, int(j), 1).view(np.uint64)[0]


def test_new_variants_every_config(gpu_lib):
    key = int(gpu_lib.make_keys(25, 1)[0])
    n = 2 * 152 * 512 * 16 + 7
    w2 = oracle.uniform2_f32(key, 5, n).view(np.uint32)
    w64 = oracle.uniform_f64(key, 5, n).view(np.uint64)
    try:
        for v in range(C.sq_num_variants(C.SQ_KERNEL_UNIFORM2_F32)):
            C.sq_set_config(C.SQ_KERNEL_UNIFORM2_F32, 0, v, 256, 0)
            C.sq_set_config(C.SQ_KERNEL_UNIFORM_F64, 0, v, 512, 0)
            assert np.array_equal(_run(C.sq_uniform2_f32, 4, np.float32, key, 5, n=n, off=2).view(np.uint32), w2)
            assert np.array_equal(_run(C.sq_uniform2_f32, 4, np.float32, key, 5, n=n, off=1).view(np.uint32), w2)
            assert np.array_equal(_run(C.sq_uniform_f64, 8, np.float64, key, 5, n=n, off=1).view(np.uint64), w64)
    finally:
        C.sq_set_config(C.SQ_KERNEL_UNIFORM2_F32, 0, 0, 256, 0)
        C.sq_set_config(C.SQ_KERNEL_UNIFORM_F64, 0, 0, 256, 0)
