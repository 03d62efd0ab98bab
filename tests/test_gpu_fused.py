"""GPU parity of the generation-only statistics (sq_fused_stats) against the
oracle: per-stream XOR and top-byte sums bit for bit, the 256-bin top-byte
histogram exactly, for stream counts and lengths that exercise the split of
streams into parts."""
import numpy as np
import pytest

import oracle
from paper_2004_06278_gb300 import _lib as C
from tests.gpu_util import stream_handle, to_dev

pytestmark = pytest.mark.gpu


def _run(gpu_lib, keys_np, bases_np, cps):
    import torch

    S = keys_np.size
    keys, bases = to_dev(keys_np), to_dev(bases_np)
    xor = torch.empty(max(S, 1), dtype=torch.int32, device="cuda")
    sums = torch.empty(max(S, 1), dtype=torch.int64, device="cuda")
    hist = torch.full((256,), -1, dtype=torch.int64, device="cuda")
    C.sq_fused_stats(keys.data_ptr(), bases.data_ptr(), S, cps, xor.data_ptr(), sums.data_ptr(),
                     hist.data_ptr(), stream_handle())
    torch.cuda.synchronize()
    return (xor.cpu().numpy().view(np.uint32)[:S], sums.cpu().numpy().view(np.uint64)[:S],
            hist.cpu().numpy().view(np.uint64))


@pytest.mark.parametrize("S,cps", [(1, 1), (1, 31), (3, 1000), (1, 1 << 20), (7, 300_001),
                                   (1000, 64), (5000, 2048), (1 << 16, 33)])
def test_fused_matches_oracle(gpu_lib, S, cps):
    rng = np.random.default_rng(S * 7 + cps)
    keys = gpu_lib.make_keys(13, S)
    bases = rng.integers(0, 1 << 64, S, dtype=np.uint64)
    bases[::5] = np.uint64((1 << 64) - 17)  # some streams wrap
    x, s, h = _run(gpu_lib, keys, bases, cps)
    ex, es, eh = oracle.fused_stats(oracle.make_keys(13, S), bases, cps)
    assert np.array_equal(x, ex)
    assert np.array_equal(s, es)
    assert np.array_equal(h, eh)


def test_fused_zero_counters_clears_outputs(gpu_lib):
    keys = gpu_lib.make_keys(13, 10)
    x, s, h = _run(gpu_lib, keys, np.zeros(10, dtype=np.uint64), 0)
    assert not x.any() and not s.any() and not h.any()


@pytest.mark.parametrize("S,cps", [(1, 5000), (2, (1 << 20) + 3), (700, 1)])
def test_fused_both_item_layouts(gpu_lib, S, cps):
    """CTA items (variant 0) and warp items (variant 1) give the oracle's
    statistics on few long streams (split into many parts) and on many
    one-counter streams (most threads of a CTA idle)."""
    rng = np.random.default_rng(S + cps)
    keys = gpu_lib.make_keys(15, S)
    bases = rng.integers(0, 1 << 64, S, dtype=np.uint64)
    ex, es, eh = oracle.fused_stats(oracle.make_keys(15, S), bases, cps)
    try:
        for v in (0, 1):
            C.sq_set_config(C.SQ_KERNEL_FUSED, 0, v, 256, 0)
            x, s, h = _run(gpu_lib, keys, bases, cps)
            assert np.array_equal(x, ex) and np.array_equal(s, es) and np.array_equal(h, eh), v
    finally:
        C.sq_set_config(C.SQ_KERNEL_FUSED, 0, 0, 256, 0)


def test_fused_every_launch_config(gpu_lib):
    S, cps = 300, 5000
    keys = gpu_lib.make_keys(14, S)
    bases = np.arange(S, dtype=np.uint64) * np.uint64(1 << 40)
    ex, es, eh = oracle.fused_stats(oracle.make_keys(14, S), bases, cps)
    try:
        for v in range(C.sq_num_variants(C.SQ_KERNEL_FUSED)):
            for block in (128, 256, 512):
                for ctas in (1, 2, 0):
                    C.sq_set_config(C.SQ_KERNEL_FUSED, 0, v, block, ctas)
                    x, s, h = _run(gpu_lib, keys, bases, cps)
                    assert np.array_equal(x, ex) and np.array_equal(s, es) and np.array_equal(h, eh), (v, block, ctas)
    finally:
        C.sq_set_config(C.SQ_KERNEL_FUSED, 0, 0, 256, 0)
