"""Full-size parity: every output of the benchmark workloads, generated in the
launch configuration the benchmark uses (the same autotuning calls first),
compared with the oracle chunk by chunk on the host (the oracle runs on all
host cores).

  squares64, 2^30 outputs, and squares32, 2^32 outputs, one key (seed 2),
  counter base uniform in [0, 2^64);
  squares32, 2^24 outputs from counter 0, key of seed 1;
  the ragged batch of 4096 streams (seed 7, wrapping streams), the
  mid-length (2^14 streams), short (2^20) and very short (2^22) batches,
  and one flattened-warp group at each side of its 2^31-value switch from
  32-bit to 64-bit positions;
  uniform FP32 / BF16 (exact) and normals (error bounds), 2^30 each;
  two floats per squares64 output and 53-bit doubles, 2^30 each; strided
  counters, 2^30 squares32 and squares64; key-counter mode over 2^27 keys;
  generation-only statistics, 2^20 streams x 2^18 counters.
"""
import numpy as np
import pytest

import oracle
from paper_2004_06278_gb300 import _lib as C
from paper_2004_06278_gb300 import workloads
from tests.gpu_util import stream_handle, to_dev
from tests.test_gpu_transforms import ABS_TOL, REL_TOL, normal_errors

pytestmark = pytest.mark.gpu

CHUNK = 1 << 27  # elements compared per step


def _compare_chunks(dev_tensor, n, expect_fn, np_dtype):
    import torch

    torch.cuda.synchronize()
    for a in range(0, n, CHUNK):
        b = min(n, a + CHUNK)
        got = dev_tensor[a:b].cpu().numpy().view(np_dtype)
        want = expect_fn(a, b - a)
        if not np.array_equal(got, want):
            bad = np.nonzero(got != want)[0]
            raise AssertionError(f"mismatch at {a + int(bad[0])}: {got[bad[0]]} != {want[bad[0]]}"
                                 f" ({bad.size} in chunk)")


def test_u64_2p30_all_outputs(gpu_lib):
    import torch

    key = int(gpu_lib.make_keys(2, 1)[0])
    base = workloads.throughput_base(3)
    n = 1 << 30
    C.sq_autotune(C.SQ_KERNEL_U64, n)  # as bench.py does
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    C.sq_u64(key, base, n, out.data_ptr(), stream_handle())
    _compare_chunks(out, n, lambda a, m: oracle.fill64(key, (base + a) % (1 << 64), m), np.uint64)
    del out
    torch.cuda.empty_cache()


def test_u32_2p32_all_outputs(gpu_lib):
    import torch

    key = int(gpu_lib.make_keys(2, 1)[0])
    base = workloads.throughput_base(3)
    n = 1 << 32
    C.sq_autotune(C.SQ_KERNEL_U32, n)  # as bench.py does
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    C.sq_u32(key, base, n, out.data_ptr(), stream_handle())
    _compare_chunks(out, n, lambda a, m: oracle.fill32(key, (base + a) % (1 << 64), m), np.uint32)
    del out
    torch.cuda.empty_cache()


def test_batched_4096_all_outputs(gpu_lib):
    import torch

    b = workloads.ragged_batch(4096, seed=7)
    assert b.total > 4_000_000_000
    wrapping = [s for s in range(b.nstreams)
                if int(b.bases[s]) + int(b.lengths[s]) > (1 << 64)]
    assert len(wrapping) == 64
    keys_dev = gpu_lib.make_keys(b.key_seed, b.nstreams)
    keys_or = oracle.make_keys(b.key_seed, b.nstreams)
    out = torch.empty(b.total, dtype=torch.int32, device="cuda")
    # keep the device inputs referenced until the kernel has run
    d_keys, d_bases = to_dev(keys_dev), to_dev(b.bases)
    d_lengths, d_offsets = to_dev(b.lengths), to_dev(b.offsets)
    C.sq_autotune_batch(d_keys.data_ptr(), d_bases.data_ptr(), d_lengths.data_ptr(),
                        d_offsets.data_ptr(), b.nstreams, out.data_ptr())  # as bench.py does
    out.fill_(0)
    C.sq_batch(d_keys.data_ptr(), d_bases.data_ptr(), d_lengths.data_ptr(), d_offsets.data_ptr(),
               b.nstreams, out.data_ptr(), stream_handle())

    def expect(a, m):
        """The oracle's batch restricted to positions [a, a + m): the streams
        that meet the window, each clipped to it (its counter base advanced
        by the clipped prefix), in one call."""
        ends = b.offsets + b.lengths
        sel = np.nonzero((b.offsets < a + m) & (ends > a))[0]
        lo = np.maximum(b.offsets[sel], a)
        hi = np.minimum(ends[sel], a + m)
        bases = b.bases[sel] + (lo - b.offsets[sel]).astype(np.uint64)  # wraps modulo 2^64
        res = np.zeros(m, dtype=np.uint32)
        oracle.batch32(keys_or[sel], bases, (hi - lo).astype(np.int64), (lo - a).astype(np.int64), res)
        return res

    _compare_chunks(out, b.total, expect, np.uint32)
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("S,lo,hi", [(1 << 14, 3e3, 3e4), (1 << 20, 30, 300), (1 << 22, 3, 30)])
def test_batched_regimes_all_outputs(gpu_lib, S, lo, hi):
    """The mid-length, short and very short stream batches of the
    benchmark's breakdown, in the configuration the batch tuner picks for
    each (as measured: a tile kernel with 64-thread CTAs, then flattened
    warps): every output against the oracle's batch, which also leaves
    uncovered positions untouched."""
    import torch

    b = workloads.ragged_batch(S, seed=7, lo=lo, hi=hi)
    keys_dev = gpu_lib.make_keys(b.key_seed, b.nstreams)
    out = torch.empty(b.total, dtype=torch.int32, device="cuda")
    d_keys, d_bases = to_dev(keys_dev), to_dev(b.bases)
    d_lengths, d_offsets = to_dev(b.lengths), to_dev(b.offsets)
    saved = C.sq_get_config(C.SQ_KERNEL_BATCH, 0)
    try:
        C.sq_autotune_batch(d_keys.data_ptr(), d_bases.data_ptr(), d_lengths.data_ptr(),
                            d_offsets.data_ptr(), b.nstreams, out.data_ptr())
        out.fill_(0)
        C.sq_batch(d_keys.data_ptr(), d_bases.data_ptr(), d_lengths.data_ptr(), d_offsets.data_ptr(),
                   b.nstreams, out.data_ptr(), stream_handle())
        torch.cuda.synchronize()
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, saved.variant, saved.block, saved.ctas_per_sm)
    want = np.zeros(b.total, dtype=np.uint32)
    oracle.batch32(oracle.make_keys(b.key_seed, b.nstreams), b.bases, b.lengths, b.offsets, want)
    got = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want), int(np.nonzero(got != want)[0][0])


@pytest.mark.parametrize("total", [(1 << 31) - 1, 1 << 31])
def test_flat_warp_position_widths(gpu_lib, total):
    """One warp-group of the flattened-warp kernel holding 2^31 - 1 values
    (its largest 32-bit walk) and 2^31 values (its smallest 64-bit walk):
    stream 0 of length total - 31 from a counter 2^30 below 2^64 (so it
    wraps), then 31 streams of one value each. Every output against the
    oracle, and the 64 words past the extent untouched."""
    import torch

    from tests.gpu_util import filled_u32

    S = 32
    keys = gpu_lib.make_keys(13, S)
    rng = np.random.default_rng(13)
    bases = rng.integers(0, 1 << 64, S, dtype=np.uint64)
    bases[0] = np.uint64((1 << 64) - (1 << 30))
    lengths = np.ones(S, dtype=np.int64)
    lengths[0] = total - 31
    offsets = np.zeros(S, dtype=np.int64)
    offsets[1:] = lengths[0] + np.arange(S - 1)
    fill = 0xA5A5A5A5
    out = filled_u32(total + 64, fill)
    d_keys, d_bases, d_lengths, d_offsets = to_dev(keys), to_dev(bases), to_dev(lengths), to_dev(offsets)
    flat = [v for v in range(C.sq_num_variants(C.SQ_KERNEL_BATCH))
            if C.sq_variant_name(C.SQ_KERNEL_BATCH, v) == "flat-warp"][0]
    saved = C.sq_get_config(C.SQ_KERNEL_BATCH, 0)
    try:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, flat, 256, 0)
        C.sq_batch(d_keys.data_ptr(), d_bases.data_ptr(), d_lengths.data_ptr(), d_offsets.data_ptr(),
                   S, out.data_ptr(), stream_handle())
        torch.cuda.synchronize()
    finally:
        C.sq_set_config(C.SQ_KERNEL_BATCH, 0, saved.variant, saved.block, saved.ctas_per_sm)
    k0, b0, n0 = int(keys[0]), int(bases[0]), int(lengths[0])
    _compare_chunks(out, n0, lambda a, m: oracle.fill32(k0, (b0 + a) % (1 << 64), m), np.uint32)
    tail = out[n0:].cpu().numpy().view(np.uint32)
    want = np.array([oracle.squares32(int(bases[s]), int(keys[s])) for s in range(1, S)],
                    dtype=np.uint32)
    assert np.array_equal(tail[:S - 1], want)
    assert np.all(tail[S - 1:] == fill)
    del out
    torch.cuda.empty_cache()


def test_transforms_2p30(gpu_lib):
    import torch

    key = int(gpu_lib.make_keys(11, 1)[0])
    n = 1 << 30
    for kid in (C.SQ_KERNEL_UNIFORM_F32, C.SQ_KERNEL_NORMAL_F32, C.SQ_KERNEL_UNIFORM_BF16):
        C.sq_autotune(kid, n)  # as bench.py does
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    C.sq_uniform_f32(key, 0, n, out.data_ptr(), stream_handle())
    _compare_chunks(out, n, lambda a, m: oracle.uniform_f32(key, a, m).view(np.uint32), np.uint32)
    C.sq_normal_f32(key, 0, n, out.data_ptr(), stream_handle())
    torch.cuda.synchronize()
    worst_abs, worst_rel, tails, zmax = 0.0, 0.0, 0, 0.0
    for a in range(0, n, CHUNK):
        m = min(CHUNK, n - a)
        got = out[a:a + m].cpu().numpy().view(np.float32)
        want = oracle.normal_f64(key, a // 2, m)
        ea, er, nt = normal_errors(got, want)
        worst_abs, worst_rel, tails = max(worst_abs, ea), max(worst_rel, er), tails + nt
        zmax = max(zmax, float(np.abs(want).max()))
    # the precision report of the transforms workload (shown with pytest -s)
    print(f"\nnormal_f32, 2^30 outputs, key seed 11, base 0, against FP64: max abs error "
          f"(|z| < 5) {worst_abs:.3e}, max rel error (|z| >= 5) {worst_rel:.3e}, "
          f"{tails} values with |z| >= 5, max |z| {zmax:.4f}")
    assert worst_abs <= ABS_TOL and worst_rel <= REL_TOL, (worst_abs, worst_rel)
    assert tails > 300  # P(|z| >= 5) * 2^30 is about 615
    del out
    out16 = torch.empty(n, dtype=torch.int16, device="cuda")
    C.sq_uniform_bf16(key, 0, n, out16.data_ptr(), stream_handle())
    _compare_chunks(out16, n, lambda a, m: oracle.uniform_bf16(key, a, m), np.uint16)
    del out16
    torch.cuda.empty_cache()


def test_two_floats_and_doubles_2p30(gpu_lib):
    """Two FP32 uniforms per squares64 output and 53-bit double uniforms,
    2^30 outputs each (key of seed 11, base 0), tuned as bench.py tunes
    them: every output bit-exact against the oracle."""
    import torch

    key = int(gpu_lib.make_keys(11, 1)[0])
    n = 1 << 30
    for kid in (C.SQ_KERNEL_UNIFORM2_F32, C.SQ_KERNEL_UNIFORM_F64):
        C.sq_autotune(kid, n)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    C.sq_uniform2_f32(key, 0, n, out.data_ptr(), stream_handle())
    _compare_chunks(out, n, lambda a, m: oracle.uniform2_f32(key, a // 2, m).view(np.uint32),
                    np.uint32)
    del out
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    C.sq_uniform_f64(key, 0, n, out.data_ptr(), stream_handle())
    _compare_chunks(out, n, lambda a, m: oracle.uniform_f64(key, a, m).view(np.uint64), np.uint64)
    del out
    torch.cuda.empty_cache()


def test_strided_2p30(gpu_lib):
    """Strided counters as the benchmark times them (key of seed 11, base 5,
    stride 3), 2^30 squares32 and 2^30 squares64 outputs: every output
    against the oracle."""
    import torch

    key = int(gpu_lib.make_keys(11, 1)[0])
    n, base, stride = 1 << 30, 5, 3
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    C.sq_u32_strided(key, base, stride, n, out.data_ptr(), stream_handle())
    _compare_chunks(out, n, lambda a, m: oracle.fill32_strided(key, base + a * stride, stride, m),
                    np.uint32)
    del out
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    C.sq_u64_strided(key, base, stride, n, out.data_ptr(), stream_handle())
    _compare_chunks(out, n, lambda a, m: oracle.fill64_strided(key, base + a * stride, stride, m),
                    np.uint64)
    del out
    torch.cuda.empty_cache()


def test_key_counter_2p27_keys(gpu_lib):
    """Key-counter mode as the benchmark times it: 2^27 keys (the 2^22 keys
    of seed 17, tiled 32 times) at counter 0, squares32 and squares64, every
    output against the oracle."""
    import torch

    nk = 1 << 27
    keys = np.tile(gpu_lib.make_keys(17, 1 << 22), nk >> 22)
    d_keys = to_dev(keys)
    zeros = np.zeros(CHUNK, dtype=np.uint64)
    out = torch.empty(nk, dtype=torch.int32, device="cuda")
    C.sq_keys_u32(d_keys.data_ptr(), nk, 0, out.data_ptr(), stream_handle())
    _compare_chunks(out, nk, lambda a, m: oracle.pairs32(zeros[:m], keys[a:a + m]), np.uint32)
    del out
    out = torch.empty(nk, dtype=torch.int64, device="cuda")
    C.sq_keys_u64(d_keys.data_ptr(), nk, 0, out.data_ptr(), stream_handle())
    _compare_chunks(out, nk, lambda a, m: oracle.pairs64(zeros[:m], keys[a:a + m]), np.uint64)
    del out, d_keys
    torch.cuda.empty_cache()


def test_fused_2p20_streams_2p18_counters(gpu_lib):
    import torch

    S, cps = 1 << 20, 1 << 18
    keys_dev = gpu_lib.make_keys(13, S)
    keys_or = oracle.make_keys(13, S)
    bases = np.zeros(S, dtype=np.uint64)
    xor = torch.empty(S, dtype=torch.int32, device="cuda")
    sums = torch.empty(S, dtype=torch.int64, device="cuda")
    hist = torch.empty(256, dtype=torch.int64, device="cuda")
    d_keys, d_bases = to_dev(keys_dev), to_dev(bases)
    C.sq_fused_stats(d_keys.data_ptr(), d_bases.data_ptr(), S, cps, xor.data_ptr(),
                     sums.data_ptr(), hist.data_ptr(), stream_handle())
    torch.cuda.synchronize()
    x = xor.cpu().numpy().view(np.uint32)
    s = sums.cpu().numpy().view(np.uint64)
    h = hist.cpu().numpy().view(np.uint64)
    ex, es, eh = oracle.fused_stats(keys_or, bases, cps)
    assert np.array_equal(x, ex)
    assert np.array_equal(s, es)
    assert np.array_equal(h, eh)
    assert int(h.sum()) == S * cps
