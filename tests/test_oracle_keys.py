"""Pins of the "different digits" key construction (Section 3) in the oracle:
the properties the paper states, plus the readings fixed where it is silent
(hex digits from 1..15, odd last digit, no duplicate keys). CPU only."""
import numpy as np

import oracle
from tests import pins


def _nibbles(keys: np.ndarray) -> np.ndarray:
    """(n, 16) array of hex digits, most significant first."""
    k = keys.astype(np.uint64)
    cols = [((k >> np.uint64(4 * p)) & np.uint64(0xF)).astype(np.int64) for p in range(15, -1, -1)]
    return np.stack(cols, axis=1)


def test_digit_properties():
    keys = oracle.make_keys(7, 4096)
    d = _nibbles(keys)
    assert (d != 0).all(), "digits are non-zero"
    for row in d:
        assert len(set(row[:8])) == 8, "upper eight digits differ"
        assert len(set(row[8:])) == 8, "lower eight digits differ"
    assert (d[:, 15] % 2 == 1).all(), "last digit odd: ctr*key has period 2^64"
    assert (keys % np.uint64(2) == 1).all()


def test_keys_distinct_and_prefix_stable():
    a = oracle.make_keys(11, 1 << 16)
    assert np.unique(a).size == a.size
    assert np.array_equal(oracle.make_keys(11, 1000), a[:1000])
    assert not np.array_equal(oracle.make_keys(12, 1000), a[:1000])
    assert np.array_equal(oracle.make_keys(11, 0), a[:0])


def test_digits_uniform_and_half_ones():
    """Digits are "chosen randomly" and keys have "roughly half ones": each
    position is uniform over its alphabet, and the mean popcount is
    15 * (32/15) + 2.5 = 34.5 (digits 1..15 carry 32 one-bits in total; the
    eight odd digits carry 20)."""
    keys = oracle.make_keys(5, 1 << 16)
    d = _nibbles(keys)
    for p in range(15):
        h = np.bincount(d[:, p], minlength=16)[1:]
        assert abs(pins.chi2_dev(h, keys.size)) < 6.0, p
    h = np.bincount(d[:, 15], minlength=16)[1::2]
    assert abs(pins.chi2_dev(h, keys.size)) < 6.0
    pop = np.array([bin(int(k)).count("1") for k in keys])
    assert abs(pop.mean() - 34.5) < 0.06


def test_splitmix_weyl_structure():
    """splitmix64 advances its state by a fixed odd increment gamma before
    mixing, so seeding at s + gamma shifts the sequence by one, and the
    first output for seed -gamma is mix(0) = 0 (Steele, Lea, Flood 2014)."""
    gamma = 0x9E3779B97F4A7C15
    a = oracle.splitmix64(123, 10)
    b = oracle.splitmix64(123 + gamma, 9)
    assert np.array_equal(a[1:], b)
    assert int(oracle.splitmix64((-gamma) % (1 << 64), 1)[0]) == 0
    x = oracle.splitmix64(1, 1 << 16).view(np.uint8)
    assert abs(pins.chi2_dev(np.bincount(x, minlength=256), x.size)) < 6.0


def test_key_counter_mode_uniform():
    """Section 4: counter fixed (even at 0), keys from the utility vary; the
    first outputs of the streams taken together look random."""
    keys = oracle.make_keys(17, 1 << 16)
    for ctr in (0, 1):
        out = oracle.pairs64(np.full(keys.size, ctr, dtype=np.uint64), keys)
        b = out.view(np.uint8)
        assert abs(pins.chi2_dev(np.bincount(b, minlength=256), b.size)) < 6.0
