"""GPU parity of the plain generators through the C ABI: sq_u32 (Section 2),
sq_u64 (Section 5), bit for bit against the oracle, at ragged sizes, every
alignment offset, wrapping counter bases, odd and degenerate keys, and every
launch variant."""
import numpy as np
import pytest

import oracle
from paper_2004_06278_gb300 import _lib as C
from tests.gpu_util import Guarded, stream_handle

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1
SIZES = [1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 33, 127, 1000, 4097, 65537, (1 << 20) + 3]


def _run(fn, elem, key, base, n, offset_elems=0):
    g = Guarded(n * elem, offset_elems * elem)
    fn(key, base, n, g.ptr, stream_handle())
    assert g.guards_intact(), "write outside [out, out + n)"
    return g.payload({4: np.uint32, 8: np.uint64}[elem])


def test_single_stream_2p24_seed1(gpu_lib):
    """2^24 counters from 0 with the first key of seed 1, all outputs."""
    key = int(gpu_lib.make_keys(1, 1)[0])
    n = 1 << 24
    got = _run(C.sq_u32, 4, key, 0, n)
    assert np.array_equal(got, oracle.fill32(key, 0, n))


@pytest.mark.parametrize("n", SIZES)
def test_u32_sizes_and_offsets(gpu_lib, n):
    key = int(gpu_lib.make_keys(3, 1)[0])
    base = 0x123456789ABCDEF0
    want = oracle.fill32(key, base, n)
    for off in range(8):
        assert np.array_equal(_run(C.sq_u32, 4, key, base, n, off), want), (n, off)


@pytest.mark.parametrize("n", SIZES)
def test_u64_sizes_and_offsets(gpu_lib, n):
    key = int(gpu_lib.make_keys(4, 1)[0])
    base = 0xFEDCBA9876543210
    want = oracle.fill64(key, base, n)
    for off in range(4):
        assert np.array_equal(_run(C.sq_u64, 8, key, base, n, off), want), (n, off)


def test_wraparound(gpu_lib):
    """Counters wrap modulo 2^64 (C semantics of the paper's uint64_t)."""
    key = int(gpu_lib.make_keys(5, 1)[0])
    for base in (M64, M64 - 6, (1 << 64) - 100_000):
        n = 300_001
        assert np.array_equal(_run(C.sq_u32, 4, key, base, n), oracle.fill32(key, base, n))
        assert np.array_equal(_run(C.sq_u64, 8, key, base, n), oracle.fill64(key, base, n))


@pytest.mark.parametrize("key", [0, 1, 2, M64, 1 << 63, 0x8000000000000001, 0x5555555555555555,
                                 0xAAAAAAAAAAAAAAAA])
def test_degenerate_keys(gpu_lib, key):
    n = 40_000
    base = 0x0123456789ABCDEF
    assert np.array_equal(_run(C.sq_u32, 4, key, base, n), oracle.fill32(key, base, n))
    assert np.array_equal(_run(C.sq_u64, 8, key, base, n), oracle.fill64(key, base, n))


def test_random_keys_and_bases(gpu_lib):
    rng = np.random.default_rng(99)
    for _ in range(12):
        key = int(rng.integers(0, 1 << 64, dtype=np.uint64))
        base = int(rng.integers(0, 1 << 64, dtype=np.uint64))
        n = int(rng.integers(1, 200_000))
        assert np.array_equal(_run(C.sq_u32, 4, key, base, n), oracle.fill32(key, base, n))
        assert np.array_equal(_run(C.sq_u64, 8, key, base, n), oracle.fill64(key, base, n))


def test_split_invariance(gpu_lib):
    """gen(base, n) == gen(base, m) ++ gen(base + m, n - m): the state is
    (key, ctr), so resuming at ctr + m continues the stream."""
    key = int(gpu_lib.make_keys(6, 1)[0])
    base = M64 - 12345
    n = 1_000_003
    whole = _run(C.sq_u32, 4, key, base, n)
    for m in (1, 3, 4097, 500_001):
        a = _run(C.sq_u32, 4, key, base, m)
        b = _run(C.sq_u32, 4, key, (base + m) & M64, n - m)
        assert np.array_equal(np.concatenate([a, b]), whole), m


@pytest.mark.parametrize("kid,fn,elem", [(C.SQ_KERNEL_U32, C.sq_u32, 4),
                                         (C.SQ_KERNEL_U64, C.sq_u64, 8)])
def test_every_launch_config(gpu_lib, kid, fn, elem):
    """Each body variant, block size and grid size gives identical bits."""
    key = int(gpu_lib.make_keys(8, 1)[0])
    base = M64 - 77
    n = 3 * 152 * 512 * 8 + 13
    want = oracle.fill32(key, base, n) if elem == 4 else oracle.fill64(key, base, n)
    try:
        for v in range(C.sq_num_variants(kid)):
            for block in (128, 256, 512):
                for ctas in (1, 2, 0):
                    C.sq_set_config(kid, 0, v, block, ctas)
                    for off in (0, 1):
                        assert np.array_equal(_run(fn, elem, key, base, n, off), want), (v, block, ctas)
    finally:
        C.sq_set_config(kid, 0, 0, 256, 0)


def test_async_on_torch_stream(gpu_lib):
    """Launches go to the caller's stream."""
    import torch

    key = int(gpu_lib.make_keys(9, 1)[0])
    s = torch.cuda.Stream()
    n = 1 << 22
    out = torch.empty(n, dtype=torch.uint32, device="cuda")
    with torch.cuda.stream(s):
        gpu_lib.u32(key, 5, n, out=out)
    s.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.fill32(key, 5, n))


def test_bulk_variant_device_and_host_memory(gpu_lib):
    """The shared-memory + bulk-copy variant on device memory, and its
    fallback to direct stores when the output is pinned host memory."""
    import torch

    key = int(gpu_lib.make_keys(10, 1)[0])
    bulk = [v for v in range(C.sq_num_variants(C.SQ_KERNEL_U32))
            if C.sq_variant_name(C.SQ_KERNEL_U32, v) == "bulk64"][0]
    n = 3 * 152 * 16 * 512 + 21
    try:
        for kid, fn, dt, ref in ((C.SQ_KERNEL_U32, C.sq_u32, torch.int32, oracle.fill32),
                                 (C.SQ_KERNEL_U64, C.sq_u64, torch.int64, oracle.fill64)):
            C.sq_set_config(kid, 0, bulk, 256, 0)
            want = ref(key, 11, n)
            for off in (0, 1, 3):
                elem = 4 if dt == torch.int32 else 8
                assert np.array_equal(_run(fn, elem, key, 11, n, off), want), off
            host = torch.empty(n, dtype=dt, pin_memory=True)
            fn(key, 11, n, host.data_ptr(), stream_handle())
            torch.cuda.synchronize()
            assert np.array_equal(host.numpy().view(want.dtype), want)
    finally:
        C.sq_set_config(C.SQ_KERNEL_U32, 0, 0, 256, 0)
        C.sq_set_config(C.SQ_KERNEL_U64, 0, 0, 256, 0)


@pytest.mark.parametrize("kid,fn,dt,ref", [(C.SQ_KERNEL_U32, C.sq_u32, "int32", oracle.fill32),
                                           (C.SQ_KERNEL_U64, C.sq_u64, "int64", oracle.fill64)])
def test_every_variant_into_pinned_host_memory(gpu_lib, kid, fn, dt, ref):
    """Outputs in pinned host memory: each configured variant (the wide and
    bulk ones are replaced by contiguous stores there) gives the oracle's
    bits, at an aligned and a misaligned start."""
    import torch

    key = int(gpu_lib.make_keys(12, 1)[0])
    n = 2 * 152 * 512 * 16 + 29
    want = ref(key, M64 - 5, n)
    host = torch.zeros(n + 8, dtype=getattr(torch, dt), pin_memory=True)
    try:
        for v in range(C.sq_num_variants(kid)):
            C.sq_set_config(kid, 0, v, 256, 0)
            for off in (0, 3):
                host.zero_()
                fn(key, M64 - 5, n, host[off:].data_ptr(), stream_handle())
                torch.cuda.synchronize()
                got = host.numpy().view(want.dtype)
                assert np.array_equal(got[off:off + n], want), (v, off)
                assert not got[:off].any() and not got[off + n:].any(), (v, off)
    finally:
        C.sq_set_config(kid, 0, 0, 256, 0)


@pytest.mark.parametrize("name", ["st32x2.cs", "bulk64"])
def test_capture_with_wide_and_bulk_variants(gpu_lib, name):
    """The launchers' output-memory query (made for the wide and bulk
    variants) is legal inside a stream capture: capture sq_u32 and sq_u64,
    replay, compare with the oracle."""
    import torch

    key = int(gpu_lib.make_keys(13, 1)[0])
    n = 3 * 152 * 512 * 16 + 5
    out32 = torch.empty(n, dtype=torch.int32, device="cuda")
    out64 = torch.empty(n, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    try:
        for kid in (C.SQ_KERNEL_U32, C.SQ_KERNEL_U64):
            v = [i for i in range(C.sq_num_variants(kid)) if C.sq_variant_name(kid, i) == name][0]
            C.sq_set_config(kid, 0, v, 256, 0)
        with torch.cuda.stream(s):
            C.sq_u32(key, 7, n, out32.data_ptr(), int(s.cuda_stream))
            C.sq_u64(key, 7, n, out64.data_ptr(), int(s.cuda_stream))
            s.synchronize()
            with torch.cuda.graph(g, stream=s):
                C.sq_u32(key, 7, n, out32.data_ptr(), int(s.cuda_stream))
                C.sq_u64(key, 7, n, out64.data_ptr(), int(s.cuda_stream))
        out32.zero_()
        out64.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out32.cpu().numpy().view(np.uint32), oracle.fill32(key, 7, n))
        assert np.array_equal(out64.cpu().numpy().view(np.uint64), oracle.fill64(key, 7, n))
    finally:
        C.sq_set_config(C.SQ_KERNEL_U32, 0, 0, 256, 0)
        C.sq_set_config(C.SQ_KERNEL_U64, 0, 0, 256, 0)


def test_fill_store_ceiling_kernel(gpu_lib):
    """sq_fill_u32 (the write-only kernel the benchmark measures the store
    ceiling with) writes exactly [out, out + n) with its value in every
    store variant and block size, at every 4-byte offset (one of them with
    a pause after each chunk), in device memory and in pinned host memory."""
    import torch

    n = 2 * 152 * 512 * 16 + 13
    value = 0x9E3779B9
    for v in range(C.sq_num_variants(C.SQ_KERNEL_U32)):
        for block in (128, 512):
            for off in (0, 1, 3, 7):
                g = Guarded(n * 4, off * 4)
                C.sq_fill_u32(value, n, g.ptr, (v, block, 0), 100 * (off == 3), stream_handle())
                assert g.guards_intact(), (v, block, off)
                assert np.all(g.payload(np.uint32) == value), (v, block, off)
    host = torch.zeros(n + 8, dtype=torch.int32, pin_memory=True)
    for off in (0, 3):
        host.zero_()
        C.sq_fill_u32(value, n, host[off:].data_ptr(), None, 0, stream_handle())
        torch.cuda.synchronize()
        got = host.numpy().view(np.uint32)
        assert np.all(got[off:off + n] == value) and not got[:off].any() and not got[off + n:].any()
