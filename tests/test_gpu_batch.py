"""GPU parity of the ragged batch (sq_batch) against the oracle: gaps and
empty streams, wrapping bases, key-counter mode (Section 4), every launch
variant, CUDA-graph capture and replay, and the debug validator."""
import numpy as np
import pytest

import oracle
from paper_2004_06278_gb300 import _lib as C
from paper_2004_06278_gb300 import workloads
from tests.gpu_util import CANARY, Guarded, filled_u32, host_u32, stream_handle, to_dev

pytestmark = pytest.mark.gpu
FILL = np.uint32(CANARY * 0x01010101)


def _device_inputs(gpu_lib, b):
    import torch

    keys = to_dev(gpu_lib.make_keys(b.key_seed, b.nstreams))
    return keys, to_dev(b.bases), to_dev(b.lengths), to_dev(b.offsets)


def _expect(b, n_out):
    out = np.full(n_out, FILL, dtype=np.uint32)
    oracle.batch32(oracle.make_keys(b.key_seed, b.nstreams), b.bases, b.lengths, b.offsets, out)
    return out


def _run(gpu_lib, b, offset_elems=0, extra=37):
    keys, bases, lengths, offsets = _device_inputs(gpu_lib, b)
    n_out = b.total + extra
    g = Guarded(4 * n_out, 4 * offset_elems)
    C.sq_batch(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(), offsets.data_ptr(),
               b.nstreams, g.ptr, stream_handle())
    assert g.guards_intact()
    return g.payload(np.uint32), n_out


@pytest.mark.parametrize("seed,S,max_len", [(1, 1, 10), (2, 5, 3), (3, 37, 3000),
                                            (4, 300, 20_000), (5, 64, 70_000), (6, 2000, 50)])
def test_small_batches(gpu_lib, seed, S, max_len):
    b = workloads.small_ragged_batch(S, seed=seed, max_len=max_len)
    for off in (0, 1, 3, 5):
        got, n_out = _run(gpu_lib, b, off)
        assert np.array_equal(got, _expect(b, n_out)), off


def test_leading_gap_and_empty_streams(gpu_lib):
    b = workloads.small_ragged_batch(50, seed=11, max_len=5000, gap_max=700)
    b.offsets = b.offsets + 12345  # nothing before offsets[0] is written
    b.lengths[[0, 7, 8, 49]] = 0
    got, n_out = _run(gpu_lib, b)
    assert np.array_equal(got, _expect(b, n_out))
    assert np.all(got[:12345] == FILL)


def test_key_counter_mode(gpu_lib):
    """Section 4: counter fixed at 0, one output per key."""
    b = workloads.key_counter_batch(1 << 16, seed=17)
    got, n_out = _run(gpu_lib, b)
    assert np.array_equal(got, _expect(b, n_out))


def test_every_launch_config(gpu_lib):
    b = workloads.small_ragged_batch(200, seed=21, max_len=40_000)
    try:
        for v in range(C.sq_num_variants(C.SQ_KERNEL_BATCH)):
            for block in (64, 128, 256, 512):
                for ctas in (1, 3, 0):
                    C.sq_set_config(C.SQ_KERNEL_BATCH, 0, v, block, ctas)
                    got, n_out = _run(gpu_lib, b, offset_elems=block % 7)
                    assert np.array_equal(got, _expect(b, n_out)), (v, block, ctas)
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, 0, 256, 0)


def _packed_batch(S, seed, lo, hi, empty=5, wrap_every=4):
    """Streams laid end to end (offsets = exclusive prefix sum of the lengths),
    a few of them empty, every wrap_every-th one wrapping at 2^64."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(lo, hi, S).astype(np.int64)
    lengths[rng.integers(0, S, empty)] = 0
    bases = rng.integers(0, 1 << 64, S, dtype=np.uint64)
    for s in range(0, S, wrap_every):
        bases[s] = np.uint64((1 << 64) - int(rng.integers(1, max(2, int(lengths[s]) + 1))))
    offsets = (np.cumsum(lengths) - lengths).astype(np.int64)
    return workloads.Batch(key_seed=seed, bases=bases, lengths=lengths, offsets=offsets)


def _seg_variants():
    segs = [v for v in range(C.sq_num_variants(C.SQ_KERNEL_BATCH))
            if C.sq_variant_name(C.SQ_KERNEL_BATCH, v).startswith("flat-seg")]
    assert len(segs) == 3
    return segs


@pytest.mark.parametrize("lo,hi", [(1, 4), (3, 30), (30, 300), (300, 3000)])
def test_seg_variants_on_batches(gpu_lib, lo, hi):
    """The flattened-warp segment variants (flat-seg4, -seg8, -seg16) need
    no packing: every output against the oracle on a packed batch at every
    output offset modulo 16 (the segment cuts follow the output address),
    and on a batch with gaps, in several block sizes, with one warp per 32
    streams (ctas_per_sm 0) and with a persistent grid (1 CTA per SM)."""
    b = _packed_batch(1000, seed=lo + 7, lo=lo, hi=hi)
    g = workloads.small_ragged_batch(1000, seed=hi + 7, max_len=hi, gap_max=5)
    g.lengths[::97] = 0
    try:
        for v in _seg_variants():
            for block in (64, 256, 512):
                for ctas in (0, 1):
                    C.sq_set_config(C.SQ_KERNEL_BATCH, 0, v, block, ctas)
                    for off in range(16):
                        got, n_out = _run(gpu_lib, b, offset_elems=off, extra=11)
                        assert np.array_equal(got, _expect(b, n_out)), (v, block, ctas, off)
                    got, n_out = _run(gpu_lib, g, offset_elems=block % 5)
                    assert np.array_equal(got, _expect(g, n_out)), (v, block, ctas, "gaps")
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, 0, 256, 0)


def test_seg_variants_long_stream_group(gpu_lib):
    """A group holding a stream of 2^26 values or more takes the
    per-position walk, the next group the segment walk, in one launch."""
    b = _packed_batch(40, seed=99, lo=1, hi=200, empty=2)
    b.lengths[5] = (1 << 26) + 3
    b.offsets = (np.cumsum(b.lengths) - b.lengths).astype(np.int64)
    want = _expect(b, b.total + 11)
    try:
        for v in _seg_variants():
            C.sq_set_config(C.SQ_KERNEL_BATCH, 0, v, 256, 0)
            got, n_out = _run(gpu_lib, b, offset_elems=3, extra=11)
            assert np.array_equal(got, want), v
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, 0, 256, 0)


def test_batch_equals_plain_per_stream(gpu_lib):
    import torch

    b = workloads.ragged_batch(64, seed=23, lo=1e3, hi=3e5)
    got, _ = _run(gpu_lib, b)
    keys = gpu_lib.make_keys(b.key_seed, b.nstreams)
    for s in range(b.nstreams):
        n = int(b.lengths[s])
        plain = gpu_lib.u32(int(keys[s]), int(b.bases[s]), n).cpu().numpy()
        a = int(b.offsets[s])
        assert np.array_equal(got[a:a + n], plain), s
    torch.cuda.synchronize()


@pytest.mark.parametrize("variant", ["st32", "flat-warp", "flat-seg8"])
def test_torch_graph_capture_and_replay(gpu_lib, variant):
    """The launch is capture-safe: capture once, change lengths/offsets/bases
    on the device, replay, and get the new batch; for the tile kernel and
    for the flattened-warp kernels (whose grid follows the stream count,
    known on the host)."""
    import torch

    b1 = workloads.small_ragged_batch(100, seed=31, max_len=10_000)
    b2 = workloads.small_ragged_batch(100, seed=32, max_len=10_000)
    b2.key_seed = b1.key_seed
    n_out = max(b1.total, b2.total) + 11
    keys, bases, lengths, offsets = _device_inputs(gpu_lib, b1)
    out = filled_u32(n_out, int(FILL))
    v = [i for i in range(C.sq_num_variants(C.SQ_KERNEL_BATCH))
         if C.sq_variant_name(C.SQ_KERNEL_BATCH, i) == variant][0]
    C.sq_set_config(C.SQ_KERNEL_BATCH, b1.nstreams, v, 128, 0)
    try:
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            gpu_lib.batch(keys, bases, lengths, offsets, out)  # warm-up outside capture
            s.synchronize()
            with torch.cuda.graph(g, stream=s):
                gpu_lib.batch(keys, bases, lengths, offsets, out)
        out.copy_(filled_u32(n_out, int(FILL)))
        g.replay()
        assert np.array_equal(host_u32(out), _expect(b1, n_out))
        bases.copy_(to_dev(b2.bases))
        lengths.copy_(to_dev(b2.lengths))
        offsets.copy_(to_dev(b2.offsets))
        out.copy_(filled_u32(n_out, int(FILL)))
        for _ in range(3):
            g.replay()
        assert np.array_equal(host_u32(out), _expect(b2, n_out))
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, b1.nstreams, 0, 256, 0)


def test_native_graph_helper(gpu_lib):
    import torch

    b = workloads.small_ragged_batch(80, seed=41, max_len=20_000)
    keys, bases, lengths, offsets = _device_inputs(gpu_lib, b)
    n_out = b.total + 3
    out = filled_u32(n_out, int(FILL))
    torch.cuda.synchronize()
    graph = C.sq_batch_graph_create(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(),
                                    offsets.data_ptr(), b.nstreams, out.data_ptr())
    try:
        for _ in range(4):
            C.sq_graph_launch(graph, stream_handle())
        assert np.array_equal(host_u32(out), _expect(b, n_out))
    finally:
        C.sq_graph_destroy(graph)


def test_validate(gpu_lib):
    import torch

    b = workloads.small_ragged_batch(20, seed=51, max_len=100)
    _, _, lengths, offsets = _device_inputs(gpu_lib, b)
    C.sq_batch_validate(lengths.data_ptr(), offsets.data_ptr(), b.nstreams, stream_handle())
    bad = b.offsets.copy()
    bad[5] = bad[4] + b.lengths[4] - 1 if b.lengths[4] > 0 else bad[4] - 1
    offsets.copy_(to_dev(bad))
    with pytest.raises(C.SquaresError) as e:
        C.sq_batch_validate(lengths.data_ptr(), offsets.data_ptr(), b.nstreams, stream_handle())
    assert e.value.status == C.SQ_EINVAL
    neg = b.lengths.copy()
    neg[3] = -1
    lengths.copy_(to_dev(neg))
    offsets.copy_(to_dev(b.offsets))
    with pytest.raises(C.SquaresError):
        C.sq_batch_validate(lengths.data_ptr(), offsets.data_ptr(), b.nstreams, stream_handle())


def test_every_variant_into_pinned_host_memory(gpu_lib):
    """A batch written to pinned host memory (the wide variants are replaced
    by contiguous stores there) matches the oracle, canaries intact."""
    import torch

    b = workloads.small_ragged_batch(150, seed=43, max_len=30_000)
    keys, bases, lengths, offsets = _device_inputs(gpu_lib, b)
    n_out = b.total + 19
    want = _expect(b, n_out)
    host = torch.empty(n_out + 8, dtype=torch.int32, pin_memory=True)
    try:
        for v in range(C.sq_num_variants(C.SQ_KERNEL_BATCH)):
            C.sq_set_config(C.SQ_KERNEL_BATCH, 0, v, 256, 0)
            for off in (0, 5):
                host.numpy().view(np.uint32)[:] = FILL
                C.sq_batch(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(), offsets.data_ptr(),
                           b.nstreams, host[off:].data_ptr(), stream_handle())
                torch.cuda.synchronize()
                got = host.numpy().view(np.uint32)
                assert np.array_equal(got[off:off + n_out], want), (v, off)
                assert np.all(got[:off] == FILL) and np.all(got[off + n_out:] == FILL), (v, off)
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, 0, 256, 0)


def test_capture_with_wide_variant(gpu_lib):
    """The output-memory query made for the wide variants is legal inside a
    stream capture: capture with the widest variant and replay."""
    import torch

    b = workloads.small_ragged_batch(60, seed=47, max_len=20_000)
    keys, bases, lengths, offsets = _device_inputs(gpu_lib, b)
    n_out = b.total + 7
    out = filled_u32(n_out, int(FILL))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    try:
        wide = [v for v in range(C.sq_num_variants(C.SQ_KERNEL_BATCH))
                if C.sq_variant_name(C.SQ_KERNEL_BATCH, v) == "st32x2.cs"][0]
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, wide, 256, 0)
        with torch.cuda.stream(s):
            gpu_lib.batch(keys, bases, lengths, offsets, out)
            s.synchronize()
            with torch.cuda.graph(g, stream=s):
                gpu_lib.batch(keys, bases, lengths, offsets, out)
        out.copy_(filled_u32(n_out, int(FILL)))
        g.replay()
        assert np.array_equal(host_u32(out), _expect(b, n_out))
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, 0, 256, 0)


def test_capture_flat_warp_and_replay_with_new_lengths(gpu_lib):
    """The flattened-warp variant (launched with dynamic shared memory)
    captured in a CUDA graph: replayed as captured, then again after the
    lengths were halved on the device, it writes each batch exactly, since
    the kernel reads the metadata and the extent when it runs."""
    import types

    import torch

    b = workloads.small_ragged_batch(700, seed=49, max_len=40)
    keys, bases, lengths, offsets = _device_inputs(gpu_lib, b)
    n_out = b.total + 9
    out = filled_u32(n_out, int(FILL))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    flat = [v for v in range(C.sq_num_variants(C.SQ_KERNEL_BATCH))
            if C.sq_variant_name(C.SQ_KERNEL_BATCH, v) == "flat-warp"][0]
    try:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, flat, 128, 0)
        with torch.cuda.stream(s):
            gpu_lib.batch(keys, bases, lengths, offsets, out)
            s.synchronize()
            with torch.cuda.graph(g, stream=s):
                gpu_lib.batch(keys, bases, lengths, offsets, out)
        out.copy_(filled_u32(n_out, int(FILL)))
        g.replay()
        assert np.array_equal(host_u32(out), _expect(b, n_out))
        half = (b.lengths // 2).astype(np.int64)
        lengths.copy_(to_dev(half))
        out.copy_(filled_u32(n_out, int(FILL)))
        g.replay()
        b2 = types.SimpleNamespace(key_seed=b.key_seed, nstreams=b.nstreams, bases=b.bases,
                                   lengths=half, offsets=b.offsets)
        assert np.array_equal(host_u32(out), _expect(b2, n_out))
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, 0, 256, 0)


def _invalid_batches(rng):
    """Metadata that breaks sq_batch's requirements in four ways: unsorted
    offsets, streams overlapping the next ones, negative offsets, and an
    early stream reaching far past the last one's end."""
    out = []
    for kind in range(4):
        S = 24
        lengths = rng.integers(0, 400, S).astype(np.int64)
        if kind == 0:
            offsets = rng.integers(0, 3000, S).astype(np.int64)
        elif kind == 1:
            offsets = np.sort(rng.integers(0, 2000, S)).astype(np.int64)
            lengths = rng.integers(0, 4000, S).astype(np.int64)
        elif kind == 2:
            offsets = rng.integers(-500, 2000, S).astype(np.int64)
            offsets[-1] = abs(int(offsets[-1]))
        else:
            offsets = np.sort(rng.integers(0, 500, S)).astype(np.int64)
            lengths = rng.integers(0, 50, S).astype(np.int64)
            lengths[0] = 100_000
        out.append((offsets, lengths))
    return out


def test_invalid_metadata_stays_inside_the_extent(gpu_lib):
    """Whatever the offsets, no variant writes outside [0, offsets[S-1] +
    lengths[S-1]): a buffer of exactly that many elements keeps its guard
    bytes on both sides (the values inside are not defined)."""
    rng = np.random.default_rng(71)
    try:
        for offsets, lengths in _invalid_batches(rng):
            S = offsets.size
            end = int(offsets[-1] + lengths[-1])
            keys = to_dev(gpu_lib.make_keys(72, S))
            bases = to_dev(rng.integers(0, 1 << 64, S, dtype=np.uint64))
            d_len, d_off = to_dev(lengths), to_dev(offsets)
            for v in range(C.sq_num_variants(C.SQ_KERNEL_BATCH)):
                for block in (128, 512):
                    C.sq_set_config(C.SQ_KERNEL_BATCH, 0, v, block, 0)
                    for off in (0, 3):
                        g = Guarded(4 * end, 4 * off)
                        C.sq_batch(keys.data_ptr(), bases.data_ptr(), d_len.data_ptr(), d_off.data_ptr(),
                                   S, g.ptr, stream_handle())
                        assert g.guards_intact(), (v, block, off, end)
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, 0, 256, 0)
