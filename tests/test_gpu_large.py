"""GPU parity beyond 32-bit element counts: one sq_u32 launch of more than
2^32 outputs, one sq_u64 launch of more than 2^31, a ragged batch whose
middle stream alone holds more than 2^32 outputs, and generation-only
statistics over more than 2^32 counters per stream (which the launcher
splits into parts). Counter bases are chosen so that counters wrap modulo
2^64 inside each run. Outputs are compared with the oracle at sampled
positions, over whole regions at both ends and around index 2^32, and over
whole small streams; the statistics in full."""
import numpy as np
import pytest

import oracle
from paper_2004_06278_gb300 import _lib as C
from paper_2004_06278_gb300 import workloads
from tests.gpu_util import filled_u32, stream_handle, to_dev

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1
CANARY = 0xA5A5A5A5


def _at(t, idx: np.ndarray) -> np.ndarray:
    """Elements of device tensor t at positions idx, as host numpy."""
    import torch

    return t.index_select(0, torch.from_numpy(idx.astype(np.int64)).cuda()).cpu().numpy()


def _ctrs(base: int, idx: np.ndarray) -> np.ndarray:
    return idx.astype(np.uint64) + np.uint64(base)  # wraps modulo 2^64


def _variant(kid, name):
    return [v for v in range(C.sq_num_variants(kid)) if C.sq_variant_name(kid, v) == name][0]


@pytest.mark.parametrize("config", [("st32", 256), ("st32x2.cs", 512)])
def test_u32_more_than_2p32_outputs(gpu_lib, config):
    import torch

    key = int(gpu_lib.make_keys(71, 1)[0])
    n = (1 << 32) + (3 << 20) + 77
    base = M64 - (1 << 31)  # wraps inside the launch
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    try:
        C.sq_set_config(C.SQ_KERNEL_U32, 0, _variant(C.SQ_KERNEL_U32, config[0]), config[1], 0)
        C.sq_u32(key, base, n, out.data_ptr(), stream_handle())
        torch.cuda.synchronize()
    finally:
        C.sq_set_config(C.SQ_KERNEL_U32, 0, 0, 256, 0)
    idx = workloads.sample_positions(n, 200_000, seed=72)
    assert np.array_equal(_at(out, idx).view(np.uint32), oracle.pairs32(_ctrs(base, idx), np.uint64(key)))
    for a in ((1 << 32) - 4096, n - (1 << 22)):  # around index 2^32, and the tail
        m = min(1 << 22, n - a)
        got = out[a:a + m].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, oracle.fill32(key, (base + a) & M64, m)), a


def test_u64_more_than_2p31_outputs(gpu_lib):
    import torch

    key = int(gpu_lib.make_keys(75, 1)[0])
    n = (1 << 31) + (1 << 20) + 5
    base = M64 - (1 << 30)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    C.sq_u64(key, base, n, out.data_ptr(), stream_handle())
    torch.cuda.synchronize()
    idx = workloads.sample_positions(n, 200_000, seed=76)
    assert np.array_equal(_at(out, idx).view(np.uint64), oracle.pairs64(_ctrs(base, idx), np.uint64(key)))
    for a in ((1 << 31) - 4096, n - (1 << 21)):
        m = min(1 << 21, n - a)
        got = out[a:a + m].cpu().numpy().view(np.uint64)
        assert np.array_equal(got, oracle.fill64(key, (base + a) & M64, m)), a


def test_batch_stream_longer_than_2p32(gpu_lib):
    """Five streams (one empty) with gaps; the second holds 2^32 + 5000
    outputs from a base 1000 below 2^64. Gaps keep the canary."""
    import torch

    keys = gpu_lib.make_keys(73, 5)
    lengths = np.array([1000, (1 << 32) + 5000, 777, 0, 12345], dtype=np.int64)
    gaps = np.array([3, 17, 5, 0, 64], dtype=np.int64)
    offsets = np.zeros(5, dtype=np.int64)
    pos = 0
    for s in range(5):
        pos += gaps[s]
        offsets[s] = pos
        pos += lengths[s]
    n_out = pos + 11
    bases = np.array([5, M64 - 1000, 0, 9, 1 << 40], dtype=np.uint64)
    d_keys, d_bases, d_len, d_off = to_dev(keys), to_dev(bases), to_dev(lengths), to_dev(offsets)
    out = filled_u32(n_out, CANARY)
    C.sq_batch(d_keys.data_ptr(), d_bases.data_ptr(), d_len.data_ptr(), d_off.data_ptr(), 5,
               out.data_ptr(), stream_handle())
    torch.cuda.synchronize()
    for s in (0, 2, 4):  # small streams in full, with their gaps
        a, m = int(offsets[s]), int(lengths[s])
        got = out[a - int(gaps[s]):a + m].cpu().numpy().view(np.uint32)
        assert np.all(got[:int(gaps[s])] == CANARY), s
        assert np.array_equal(got[int(gaps[s]):], oracle.fill32(int(keys[s]), int(bases[s]), m)), s
    a, m = int(offsets[1]), int(lengths[1])
    idx = workloads.sample_positions(m, 200_000, seed=74)
    got = _at(out, idx + a).view(np.uint32)
    assert np.array_equal(got, oracle.pairs32(_ctrs(int(bases[1]), idx), keys[1]))
    for r in (0, (1 << 32) - 4096, m - (1 << 20)):  # head, around 2^32, tail
        k = min(1 << 20, m - r)
        got = out[a + r:a + r + k].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, oracle.fill32(int(keys[1]), (int(bases[1]) + r) & M64, k)), r
    tail = out[pos:].cpu().numpy().view(np.uint32)
    assert np.all(tail == CANARY)


def test_flattened_warp_group_past_2p31(gpu_lib):
    """The flattened-warp variants on a group of streams holding more than
    2^31 values (one stream of 2^31 + 5000): the group scan runs in 64-bit
    words, the per-position walk in 64-bit positions, and the segment
    variant hands the group to that walk; the next group, all short streams
    past output 2^31, takes the segment walk there. Sampled outputs, windows
    at the head, around 2^31 and the tail, the small streams in full, gaps
    and the tail canary."""
    import torch

    # streams 5..39 are short and follow the long one: the second group of
    # 32 (streams 32..39) takes the segment walk at outputs past 2^31
    S = 40
    keys = gpu_lib.make_keys(75, S)
    rng = np.random.default_rng(77)
    lengths = np.concatenate([[1000, (1 << 31) + 5000, 777, 0, 12345],
                              rng.integers(1, 300, S - 5)]).astype(np.int64)
    gaps = np.concatenate([[3, 17, 5, 0, 64], rng.integers(0, 4, S - 5)]).astype(np.int64)
    offsets = np.zeros(S, dtype=np.int64)
    pos = 0
    for s in range(S):
        pos += gaps[s]
        offsets[s] = pos
        pos += lengths[s]
    n_out = pos + 11
    bases = np.concatenate([np.array([5, M64 - 1000, 0, 9, 1 << 40], dtype=np.uint64),
                            rng.integers(0, 1 << 64, S - 5, dtype=np.uint64)])
    d_keys, d_bases, d_len, d_off = to_dev(keys), to_dev(bases), to_dev(lengths), to_dev(offsets)
    names = {C.sq_variant_name(C.SQ_KERNEL_BATCH, v): v for v in range(C.sq_num_variants(C.SQ_KERNEL_BATCH))}
    a, m = int(offsets[1]), int(lengths[1])
    idx = workloads.sample_positions(m, 100_000, seed=76)
    want_idx = oracle.pairs32(_ctrs(int(bases[1]), idx), keys[1])
    try:
        for name in ("flat-warp", "flat-seg8"):
            C.sq_set_config(C.SQ_KERNEL_BATCH, S, names[name], 128, 0)
            out = filled_u32(n_out, CANARY)
            C.sq_batch(d_keys.data_ptr(), d_bases.data_ptr(), d_len.data_ptr(), d_off.data_ptr(), S,
                       out.data_ptr(), stream_handle())
            torch.cuda.synchronize()
            for s in [0, 2, 4] + list(range(5, S)):
                b0, k = int(offsets[s]), int(lengths[s])
                got = out[b0 - int(gaps[s]):b0 + k].cpu().numpy().view(np.uint32)
                assert np.all(got[:int(gaps[s])] == CANARY), (name, s)
                assert np.array_equal(got[int(gaps[s]):], oracle.fill32(int(keys[s]), int(bases[s]), k)), (name, s)
            assert np.array_equal(_at(out, idx + a).view(np.uint32), want_idx), name
            for r in (0, (1 << 31) - 4096, m - (1 << 20)):
                k = min(1 << 20, m - r)
                got = out[a + r:a + r + k].cpu().numpy().view(np.uint32)
                assert np.array_equal(got, oracle.fill32(int(keys[1]), (int(bases[1]) + r) & M64, k)), (name, r)
            assert np.all(out[pos:].cpu().numpy().view(np.uint32) == CANARY), name
            del out
            torch.cuda.empty_cache()
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, S, 0, 256, 0)


def test_fused_more_than_2p32_counters_per_stream(gpu_lib):
    import torch

    keys = gpu_lib.make_keys(77, 4)
    bases = np.array([0, M64 - (1 << 31), 1 << 33, 12345], dtype=np.uint64)
    cps = (1 << 32) + 12345
    d_keys, d_bases = to_dev(keys), to_dev(bases)
    xor = torch.empty(4, dtype=torch.int32, device="cuda")
    sums = torch.empty(4, dtype=torch.int64, device="cuda")
    hist = torch.empty(256, dtype=torch.int64, device="cuda")
    C.sq_fused_stats(d_keys.data_ptr(), d_bases.data_ptr(), 4, cps, xor.data_ptr(), sums.data_ptr(),
                     hist.data_ptr(), stream_handle())
    torch.cuda.synchronize()
    ex, es, eh = oracle.fused_stats(keys, bases, cps)
    assert np.array_equal(xor.cpu().numpy().view(np.uint32), ex)
    assert np.array_equal(sums.cpu().numpy().view(np.uint64), es)
    assert np.array_equal(hist.cpu().numpy().view(np.uint64), eh)
    assert int(eh.sum()) == 4 * cps
