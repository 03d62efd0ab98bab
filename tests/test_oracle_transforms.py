"""Pins of the oracle's distribution transforms, ragged batch and fused
statistics, against library routines (numpy, scipy) and closed forms.
CPU only."""
import numpy as np
from scipy import stats

import oracle
from tests import pins

KEY = None


def key():
    global KEY
    if KEY is None:
        KEY = int(oracle.make_keys(11, 1)[0])
    return KEY


def test_uniform_f32_is_top24_over_2p24():
    n = (1 << 16) + 5
    u = oracle.fill32(key(), 77, n)
    v = oracle.uniform_f32(key(), 77, n)
    expect = (u >> 8).astype(np.float32) * np.float32(2.0 ** -24)
    assert np.array_equal(v, expect)
    assert v.min() >= 0.0 and v.max() < 1.0
    assert np.all(np.floor(v.astype(np.float64) * 2 ** 24) == v.astype(np.float64) * 2 ** 24)


def test_uniform_bf16_rounds_toward_zero():
    """bfloat16 has 8 significant bits; rounding toward zero keeps the
    largest such value not above v, so 0 <= v - b < ulp(b) and b < 1."""
    n = 1 << 16
    v = oracle.uniform_f32(key(), 5, n).astype(np.float64)
    bits = oracle.uniform_bf16(key(), 5, n)
    b = (bits.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    assert np.all(b <= v)
    nz = b > 0
    ulp = np.exp2(np.floor(np.log2(b[nz])) - 7)
    assert np.all(v[nz] - b[nz] < ulp)
    assert np.all(v[~nz] < 2.0 ** -126)
    assert b.max() < 1.0
    # on exactly representable values the conversion is the identity
    m = np.frexp(v)[0]
    exact = np.floor(m * 256) == m * 256
    assert np.array_equal(b[exact], v[exact])


def test_normal_distribution_matches_scipy():
    z = oracle.normal_f64(key(), 0, 200_001)
    assert z.size == 200_001
    d, p = stats.kstest(z, stats.norm.cdf)
    assert p > 1e-6, (d, p)
    assert abs(z.mean()) < 6 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 6 * np.sqrt(2 / z.size)
    assert abs(np.corrcoef(z[0:-1:2], z[1::2])[0, 1]) < 6 / np.sqrt(z.size / 2)


def test_normal_polar_form():
    """Inverse routes: the pair (z0, z1) from squares64 output v has radius
    sqrt(-2 ln((hi + 1) / 2^32)) and angle 2 pi lo / 2^32, with hi, lo the
    upper and lower 32 bits of v."""
    n = 4096
    v = oracle.fill64(key(), 9, n // 2)
    z = oracle.normal_f64(key(), 9, n)
    hi = (v >> np.uint64(32)).astype(np.float64)
    lo = (v & np.uint64(0xFFFFFFFF)).astype(np.float64)
    r2 = z[0::2] ** 2 + z[1::2] ** 2
    assert np.allclose(r2, -2 * np.log((hi + 1) / 2 ** 32), rtol=1e-12, atol=1e-12)
    ang = np.mod(np.arctan2(z[1::2], z[0::2]), 2 * np.pi)
    want = 2 * np.pi * lo / 2 ** 32
    dang = np.angle(np.exp(1j * (ang - want)))
    big = r2 > 1e-6
    assert np.all(np.abs(dang[big]) < 1e-9)
    # odd n drops the last sine
    z_odd = oracle.normal_f64(key(), 9, 7)
    assert np.array_equal(z_odd, z[:7])


def test_uniform53_closed_forms():
    """floor(v / 2^11) / 2^53 at points with known values, and agreement
    with numpy's exact conversion of 53-bit integers."""
    M = (1 << 64) - 1
    v = np.array([0, 2047, 2048, 1 << 63, M, (1 << 43) - 1, 1 << 43, 3 << 62], dtype=np.uint64)
    want = np.array([0.0, 0.0, 2.0 ** -53, 0.5, 1 - 2.0 ** -53, (2.0 ** 32 - 1) * 2.0 ** -53,
                     2.0 ** -21, 0.75])
    assert np.array_equal(oracle.uniform53_of(v), want)
    r = np.random.default_rng(5).integers(0, 1 << 64, 10_000, dtype=np.uint64)
    assert np.array_equal(oracle.uniform53_of(r), (r >> np.uint64(11)).astype(np.float64) * 2.0 ** -53)
    f = oracle.fill64(key(), 3, 1000)
    assert np.array_equal(oracle.uniform53_of(f), oracle.uniform_f64(key(), 3, 1000))


def test_box_muller_pairs_battery():
    """The per-halves form against closed-form points and the polar
    identities (tests/pins.py)."""
    pins.run_box_muller_battery(oracle.box_muller_f64)


def test_box_muller_pairs_match_normals():
    """On squares64 outputs the per-halves form equals the normals of those
    counters."""
    v = oracle.fill64(key(), 21, 5000)
    hi = (v >> np.uint64(32)).astype(np.uint32)
    lo = (v & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    z = oracle.box_muller_f64(hi, lo)
    assert np.array_equal(z.reshape(-1), oracle.normal_f64(key(), 21, 10_000))


def test_batch_is_concatenation_and_leaves_gaps():
    rng = np.random.default_rng(3)
    S = 9
    keys = oracle.make_keys(7, S)
    lengths = rng.integers(0, 50, S).astype(np.int64)
    gaps = rng.integers(0, 4, S).astype(np.int64)
    offsets = (np.cumsum(lengths + gaps) - lengths).astype(np.int64)
    bases = rng.integers(0, 1 << 64, S, dtype=np.uint64)
    bases[0] = np.uint64((1 << 64) - 3)  # wraps
    total = int(offsets[-1] + lengths[-1])
    out = np.full(total + 2, 0xDEADBEEF, dtype=np.uint32)
    oracle.batch32(keys, bases, lengths, offsets, out)
    mask = np.zeros(out.size, dtype=bool)
    for s in range(S):
        a, n = int(offsets[s]), int(lengths[s])
        assert np.array_equal(out[a:a + n], oracle.fill32(int(keys[s]), int(bases[s]), n))
        mask[a:a + n] = True
    assert np.all(out[~mask] == 0xDEADBEEF)


def test_fused_stats_against_numpy():
    rng = np.random.default_rng(4)
    S, C = 37, 1000
    keys = oracle.make_keys(13, S)
    bases = rng.integers(0, 1 << 64, S, dtype=np.uint64)
    bases[3] = np.uint64((1 << 64) - 10)
    x, s, h = oracle.fused_stats(keys, bases, C, threads=4)
    allv = []
    for i in range(S):
        v = oracle.fill32(int(keys[i]), int(bases[i]), C)
        allv.append(v)
        assert int(x[i]) == int(np.bitwise_xor.reduce(v))
        assert int(s[i]) == int((v >> 24).astype(np.uint64).sum())
    allv = np.concatenate(allv)
    assert np.array_equal(h, np.bincount(allv >> 24, minlength=256).astype(np.uint64))


def test_strided_is_subsampled_stream():
    """Counters base + i*stride: the same values as every stride-th output of
    the consecutive stream (and key-counter mode is stride 0 of pairs)."""
    k = key()
    base = (1 << 64) - 50
    for stride in (1, 3, 7):
        n = 1000
        assert np.array_equal(oracle.fill32_strided(k, base, stride, n),
                              oracle.fill32(k, base, n * stride)[::stride])
        assert np.array_equal(oracle.fill64_strided(k, base, stride, n),
                              oracle.fill64(k, base, n * stride)[::stride])
    same = oracle.fill32_strided(k, 99, 0, 5)
    assert np.all(same == oracle.squares32(99, k))


def test_uniform2_halves_against_numpy():
    n = 2001
    v = oracle.fill64(key(), 3, (n + 1) // 2)
    halves = np.stack([v >> np.uint64(32), v & np.uint64(0xFFFFFFFF)], axis=1).reshape(-1)[:n]
    expect = (halves >> np.uint64(8)).astype(np.float32) * np.float32(2.0 ** -24)
    assert np.array_equal(oracle.uniform2_f32(key(), 3, n), expect)


def test_uniform_f64_against_numpy():
    n = 5000
    v = oracle.fill64(key(), 11, n)
    expect = (v >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    got = oracle.uniform_f64(key(), 11, n)
    assert np.array_equal(got, expect)
    assert got.min() >= 0 and got.max() < 1
    assert np.all(np.floor(got * 2.0 ** 53) == got * 2.0 ** 53)
