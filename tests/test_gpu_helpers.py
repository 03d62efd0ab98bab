"""The torch helpers of the package (allocation + the C-ABI call on the
current stream) for every entry point, against the oracle: dtypes, shapes,
the `out=` form and a caller-given stream."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


def test_every_helper(gpu_lib):
    import torch

    key = int(gpu_lib.make_keys(95, 1)[0])
    base, n = M64 - 999, 100_001
    checks = [
        (gpu_lib.u32(key, base, n), torch.uint32, oracle.fill32(key, base, n)),
        (gpu_lib.u64(key, base, n), torch.uint64, oracle.fill64(key, base, n)),
        (gpu_lib.uniform_f32(key, base, n), torch.float32, oracle.uniform_f32(key, base, n)),
        (gpu_lib.uniform2_f32(key, base, n), torch.float32, oracle.uniform2_f32(key, base, n)),
        (gpu_lib.uniform_f64(key, base, n), torch.float64, oracle.uniform_f64(key, base, n)),
        (gpu_lib.u32_strided(key, base, 7, n), torch.uint32, oracle.fill32_strided(key, base, 7, n)),
        (gpu_lib.u64_strided(key, base, 7, n), torch.uint64, oracle.fill64_strided(key, base, 7, n)),
    ]
    for got, dt, want in checks:
        assert got.dtype == dt and got.shape == (n,) and got.is_cuda
        assert np.array_equal(got.cpu().view(torch.uint8).numpy().view(want.dtype), want)
    bf = gpu_lib.uniform_bf16(key, base, n)
    assert bf.dtype == torch.bfloat16
    assert np.array_equal(bf.cpu().view(torch.int16).numpy().view(np.uint16), oracle.uniform_bf16(key, base, n))
    z = gpu_lib.normal_f32(key, base, n)
    assert z.dtype == torch.float32
    assert np.max(np.abs(z.cpu().numpy().astype(np.float64) - oracle.normal_f64(key, base, n))) < 1e-5

    keys = gpu_lib.make_keys(96, 4099)
    d_keys = torch.from_numpy(keys.view(np.int64)).cuda()
    ctrs = np.full(keys.size, 12345, dtype=np.uint64)
    k32 = gpu_lib.keys_u32(d_keys, 12345)
    k64 = gpu_lib.keys_u64(d_keys, 12345)
    assert k32.dtype == torch.uint32 and k64.dtype == torch.uint64
    assert np.array_equal(k32.cpu().view(torch.int32).numpy().view(np.uint32), oracle.pairs32(ctrs, keys))
    assert np.array_equal(k64.cpu().view(torch.int64).numpy().view(np.uint64), oracle.pairs64(ctrs, keys))

    S, cps = 33, 5000
    fk = gpu_lib.make_keys(97, S)
    fb = np.arange(S, dtype=np.uint64) * np.uint64(1 << 40)
    xor, sums, hist = gpu_lib.fused_stats(torch.from_numpy(fk.view(np.int64)).cuda(),
                                          torch.from_numpy(fb.view(np.int64)).cuda(), cps)
    ex, es, eh = oracle.fused_stats(fk, fb, cps)
    assert np.array_equal(xor.cpu().view(torch.int32).numpy().view(np.uint32), ex)
    assert np.array_equal(sums.cpu().view(torch.int64).numpy().view(np.uint64), es)
    assert np.array_equal(hist.cpu().view(torch.int64).numpy().view(np.uint64), eh)


def test_out_and_stream_arguments(gpu_lib):
    import torch

    key = int(gpu_lib.make_keys(98, 1)[0])
    n = 4097
    s = torch.cuda.Stream()
    out = torch.zeros(n + 3, dtype=torch.uint32, device="cuda")
    r = gpu_lib.u32(key, 5, n, out=out, stream=s)
    s.synchronize()
    assert r.data_ptr() == out.data_ptr()
    got = out.cpu().view(torch.int32).numpy().view(np.uint32)
    assert np.array_equal(got[:n], oracle.fill32(key, 5, n)) and not got[n:].any()
    with pytest.raises(ValueError):
        gpu_lib.u32(key, 5, n, out=torch.zeros(n - 1, dtype=torch.uint32, device="cuda"))
