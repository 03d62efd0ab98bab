"""The autotuner on the GPU: tuned configurations give the same bits as the
oracle, the table survives a save/load round trip, and tuning the batch on
the caller's own arrays leaves correct outputs behind."""
import numpy as np
import pytest

import oracle
from paper_2004_06278_gb300 import _lib as C
from paper_2004_06278_gb300 import workloads
from tests.gpu_util import filled_u32, host_u32, stream_handle, to_dev

pytestmark = pytest.mark.gpu


def test_autotune_plain_roundtrip(gpu_lib, tmp_path):
    import torch

    n = 1 << 24
    key = int(gpu_lib.make_keys(41, 1)[0])
    try:
        for kid in (C.SQ_KERNEL_U32, C.SQ_KERNEL_U64, C.SQ_KERNEL_UNIFORM_F32):
            C.sq_autotune(kid, n)
        cfg = C.sq_get_config(C.SQ_KERNEL_U32, n)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        C.sq_u32(key, 9, n, out.data_ptr(), stream_handle())
        assert np.array_equal(host_u32(out), oracle.fill32(key, 9, n))
        path = tmp_path / "tune.txt"
        C.sq_autotune_save(str(path))
        C.sq_set_config(C.SQ_KERNEL_U32, 0, 2, 128, 1)
        C.sq_autotune_load(str(path))
        got = C.sq_get_config(C.SQ_KERNEL_U32, n)
        assert (got.variant, got.block, got.ctas_per_sm) == (cfg.variant, cfg.block, cfg.ctas_per_sm)
    finally:
        for kid in (C.SQ_KERNEL_U32, C.SQ_KERNEL_U64, C.SQ_KERNEL_UNIFORM_F32):
            C.sq_set_config(kid, 0, 0, 256, 0)


def test_autotune_batch_on_own_arrays(gpu_lib):
    b = workloads.small_ragged_batch(300, seed=43, max_len=50_000)
    keys = to_dev(gpu_lib.make_keys(b.key_seed, b.nstreams))
    bases, lengths, offsets = to_dev(b.bases), to_dev(b.lengths), to_dev(b.offsets)
    fill = 0xA5A5A5A5
    out = filled_u32(b.total + 9, fill)
    try:
        C.sq_autotune_batch(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(),
                            offsets.data_ptr(), b.nstreams, out.data_ptr())
        cfg = C.sq_get_config(C.SQ_KERNEL_BATCH, b.nstreams)
        assert 0 <= cfg.variant < C.sq_num_variants(C.SQ_KERNEL_BATCH)
        want = np.full(b.total + 9, fill, dtype=np.uint32)
        oracle.batch32(oracle.make_keys(b.key_seed, b.nstreams), b.bases, b.lengths, b.offsets, want)
        assert np.array_equal(host_u32(out), want)
        out.copy_(filled_u32(b.total + 9, fill))
        C.sq_batch(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(), offsets.data_ptr(),
                   b.nstreams, out.data_ptr(), stream_handle())
        assert np.array_equal(host_u32(out), want)
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, 0, 256, 0)


def test_autotune_batch_long_streams_keeps_tile_variants(gpu_lib):
    """With more than 8192 values per stream on average the tuner times the
    tile variants only (0-3): a per-stream lane group or warp is never
    picked there, whatever the timings. Its pick writes the batch exactly;
    the output buffer past the extent is left untouched."""
    b = workloads.small_ragged_batch(40, seed=51, max_len=60_000)
    assert b.total / b.nstreams > 8192
    keys = to_dev(gpu_lib.make_keys(b.key_seed, b.nstreams))
    bases, lengths, offsets = to_dev(b.bases), to_dev(b.lengths), to_dev(b.offsets)
    fill = 0xA5A5A5A5
    out = filled_u32(b.total + 5, fill)
    try:
        C.sq_autotune_batch(keys.data_ptr(), bases.data_ptr(), lengths.data_ptr(),
                            offsets.data_ptr(), b.nstreams, out.data_ptr())
        cfg = C.sq_get_config(C.SQ_KERNEL_BATCH, b.nstreams)
        assert 0 <= cfg.variant < 4, C.sq_variant_name(C.SQ_KERNEL_BATCH, cfg.variant)
        want = np.full(b.total + 5, fill, dtype=np.uint32)
        oracle.batch32(oracle.make_keys(b.key_seed, b.nstreams), b.bases, b.lengths, b.offsets, want)
        assert np.array_equal(host_u32(out), want)
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, 0, 256, 0)
