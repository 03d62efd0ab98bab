"""Statistical smoke tests at scale on the GPU -- cheap analogues of the
tests Section 4 lists (BigCrush and PractRand themselves are not available):
byte chi-square of one stream, counters with increments other than one,
key-counter mode (counter fixed at 0), bit-reversed words, correlation
between the streams of adjacent keys, per-bit frequencies, and three
classical tests of the kind those batteries contain (birthday spacings,
serial correlation at small lags, maximum-of-t). Each flags only
gross failures (|z| > 6). The generator is produced through the C ABI; the
histograms are counted on the device with torch."""
import numpy as np
import pytest

from paper_2004_06278_gb300 import _lib as C
from tests.gpu_util import stream_handle, to_dev
from tests.pins import chi2_dev

pytestmark = pytest.mark.gpu

N = 1 << 30


def _bytes_chi2(t):
    import torch

    counts = torch.bincount(t.view(torch.uint8).to(torch.int64), minlength=256)
    return chi2_dev(counts.cpu().numpy(), t.numel() * t.element_size())


def _bits(t):
    """Fraction of ones at each of the 32 bit positions."""
    import torch

    x = t.view(torch.int32)
    return np.array([float(((x >> b) & 1).sum().item()) / x.numel() for b in range(32)])


def _gen(fn, *args, n=N):
    import torch

    out = torch.empty(n, dtype=torch.int32, device="cuda")
    fn(*args, n, out.data_ptr(), stream_handle())
    torch.cuda.synchronize()
    return out


def test_single_stream_bytes_and_bits(gpu_lib):
    key = int(gpu_lib.make_keys(51, 1)[0])
    t = _gen(C.sq_u32, key, 0)
    assert abs(_bytes_chi2(t)) < 6
    freq = _bits(t)
    assert np.all(np.abs(freq - 0.5) < 6 * 0.5 / np.sqrt(N))


@pytest.mark.parametrize("stride", [3, (1 << 32) + 1])
def test_strided_counters(gpu_lib, stride):
    key = int(gpu_lib.make_keys(52, 1)[0])
    t = _gen(C.sq_u32_strided, key, 5, stride, n=N // 4)
    assert abs(_bytes_chi2(t)) < 6


def test_key_counter_mode_at_scale(gpu_lib):
    import torch

    keys = gpu_lib.make_keys(53, 1 << 24)
    d_keys = to_dev(keys)
    out = torch.empty(keys.size, dtype=torch.int32, device="cuda")
    C.sq_keys_u32(d_keys.data_ptr(), keys.size, 0, out.data_ptr(), stream_handle())
    torch.cuda.synchronize()
    assert abs(_bytes_chi2(out)) < 6


def test_low_bits_reversed(gpu_lib):
    """Section 4's bits-reversed test looks at the low-order bits as if they
    were the high ones. Analogues: the low 16 bits as one 65,536-bin
    histogram, and consecutive low bytes as 65,536 serial pairs."""
    import torch

    key = int(gpu_lib.make_keys(54, 1)[0])
    n = 1 << 28
    t = _gen(C.sq_u32, key, 1 << 40, n=n).view(torch.int32)
    low16 = (t & 0xFFFF).to(torch.int64)
    h = torch.bincount(low16, minlength=1 << 16)
    assert abs(chi2_dev(h.cpu().numpy(), n)) < 6
    lo8 = (t & 0xFF).to(torch.int64)
    pairs = lo8[0::2] * 256 + lo8[1::2]
    h2 = torch.bincount(pairs, minlength=1 << 16)
    assert abs(chi2_dev(h2.cpu().numpy(), n // 2)) < 6


def test_adjacent_key_streams_uncorrelated(gpu_lib):
    """Inter-stream correlation: the same counters under two consecutive
    keys from the key utility give uncorrelated uniforms, and their XOR is a
    flat byte stream."""
    import torch

    keys = gpu_lib.make_keys(55, 2)
    n = N // 4
    a = _gen(C.sq_uniform_f32, int(keys[0]), 0, n=n).view(torch.float32).double()
    b = _gen(C.sq_uniform_f32, int(keys[1]), 0, n=n).view(torch.float32).double()
    ca, cb = a - a.mean(), b - b.mean()
    corr = float((ca * cb).mean() / (ca.std() * cb.std()))
    assert abs(corr) < 6 / np.sqrt(n)
    x = _gen(C.sq_u32, int(keys[0]), 0, n=n) ^ _gen(C.sq_u32, int(keys[1]), 0, n=n)
    assert abs(_bytes_chi2(x)) < 6


def test_birthday_spacings(gpu_lib):
    """Marsaglia's birthday spacings on the 32-bit outputs: 4096 trials of
    m = 4096 birthdays in a year of 2^32 days; the number of repeated
    spacings in a trial is about Poisson(m^3 / (4 * 2^32)) = Poisson(4), so
    the total over the trials is about Poisson(16384)."""
    import torch

    key = int(gpu_lib.make_keys(56, 1)[0])
    m, trials = 4096, 4096
    t = _gen(C.sq_u32, key, 7, n=m * trials).view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    days = torch.sort(t.view(trials, m), dim=1).values
    spacings = torch.sort(days[:, 1:] - days[:, :-1], dim=1).values
    repeats = int((spacings[:, 1:] == spacings[:, :-1]).sum().item())
    lam = trials * m ** 3 / (4.0 * 2 ** 32)
    assert abs(repeats - lam) < 6 * np.sqrt(lam), (repeats, lam)


def test_serial_correlation_lags(gpu_lib):
    """Correlation of the uniforms u_i and u_{i+k} for k = 1..8 over 2^28
    values: each within 6 / sqrt(n) of zero."""
    import torch

    key = int(gpu_lib.make_keys(57, 1)[0])
    n = 1 << 28
    u = _gen(C.sq_uniform_f32, key, 0, n=n).view(torch.float32).double()
    u = u - u.mean()
    var = float((u * u).mean())
    for k in range(1, 9):
        r = float((u[:-k] * u[k:]).mean()) / var
        assert abs(r) < 6 / np.sqrt(n), (k, r)


def test_maximum_of_eight(gpu_lib):
    """Maximum-of-t with t = 8: the largest of 8 consecutive uniforms has
    distribution function x^8, so its 8th power is uniform; chi-square over
    256 equal bins of 2^25 maxima."""
    import torch

    key = int(gpu_lib.make_keys(58, 1)[0])
    groups = 1 << 25
    u = _gen(C.sq_uniform_f32, key, 11, n=8 * groups).view(torch.float32).double()
    mx = u.view(groups, 8).max(dim=1).values
    v = mx ** 8
    counts = torch.bincount(torch.clamp((v * 256).to(torch.int64), max=255), minlength=256)
    assert abs(chi2_dev(counts.cpu().numpy(), groups)) < 6


def test_squares64_bytes_and_bits(gpu_lib):
    """squares64 (Section 5): byte chi-square over 2^28 outputs and the
    frequency of ones at each of the 64 bit positions."""
    import torch

    key = int(gpu_lib.make_keys(59, 1)[0])
    n = 1 << 28
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    C.sq_u64(key, 1 << 50, n, out.data_ptr(), stream_handle())
    torch.cuda.synchronize()
    assert abs(_bytes_chi2(out)) < 6
    words = out.view(torch.int32)  # little-endian: low word, then high word
    for half in (words[0::2], words[1::2]):
        freq = _bits(half.contiguous())
        assert np.all(np.abs(freq - 0.5) < 6 * 0.5 / np.sqrt(n)), freq
