"""Pins of the generator oracle (Section 2, Section 5) against facts that do
not come from the oracle itself. CPU only."""
import numpy as np
import pytest

import oracle
from tests import pins


@pytest.fixture(scope="module")
def rng():
    return np.random.default_rng(2004_06278)


def test_hand_worked_examples():
    pins.pin_hand_worked(oracle.squares32, oracle.squares64)


def test_high_half_identity(rng):
    pins.pin_high_half(oracle.squares32, oracle.squares64, rng)


def test_zero_key():
    pins.pin_zero_key(oracle.squares32, oracle.squares64)


def test_even_key_period(rng):
    pins.pin_even_key_period(oracle.squares32, oracle.squares64, rng)


def test_odd_key_not_periodic(rng):
    pins.pin_odd_key_not_periodic(oracle.squares32, oracle.squares64, rng)


def test_z_term_enters(rng):
    pins.pin_z_term(oracle.squares32, oracle.squares64, rng)


def test_bigint_route(rng):
    pins.pin_bigint_route(oracle.squares32, oracle.squares64, rng)


def test_reduced_width_matches_full_width(rng):
    pins.pin_reduced_width_is_full_width(oracle.squares_w, oracle.squares32,
                                         oracle.squares64, rng)


def test_reduced_width_uniform_w24(rng):
    pins.pin_reduced_width_uniform(oracle.hist_w, rng, w=24, nkeys=6)


def test_reduced_width_uniform_w28(rng):
    pins.pin_reduced_width_uniform(oracle.hist_w, rng, w=28, nkeys=1)


def test_reduced_width_uniform_w32(rng):
    """32-bit state, 16-bit output: all 2^32 counters of each of three odd
    keys (chi-square within 6 sigma, every bin within 5 % of 2^16, the
    keys' histograms different) and of an even neighbour (non-uniform)."""
    pins.pin_reduced_width_uniform(oracle.hist_w, rng, w=32, nkeys=3, spread=0.05)


def test_hist_w_threads_do_not_change_it(rng):
    key = pins.reduced_keys(24, 1, rng)[0]
    assert np.array_equal(oracle.hist_w(key, 24, threads=1), oracle.hist_w(key, 24, threads=7))


def test_reduced_width_y_only_is_key_independent(rng):
    """The y-only variant (before (ctr+1)*key was added, per the
    acknowledgements) gives a histogram that does not depend on the odd key:
    with an odd key ctr -> ctr*key permutes the counters. This is the fact
    that makes ``pin_reduced_width_uniform``'s distinct-histogram check bite."""
    keys = pins.reduced_keys(20, 3, rng)
    hs = [oracle.hist_w(k, 20, 4, use_z=False) for k in keys]
    assert np.array_equal(hs[0], hs[1]) and np.array_equal(hs[0], hs[2])


def test_byte_chi2_single_stream():
    key = int(oracle.make_keys(1, 1)[0])
    pins.pin_byte_chi2(oracle.fill32, oracle.fill64, key, 0)


def test_byte_chi2_key_counter_mode():
    """Section 4's key-counter mode: counter fixed at 0, keys vary."""
    keys = oracle.make_keys(3, 1 << 18)
    out = oracle.pairs32(np.zeros(keys.size, dtype=np.uint64), keys)
    b = out.view(np.uint8)
    assert abs(pins.chi2_dev(np.bincount(b, minlength=256), b.size)) < 6.0


def test_byte_chi2_stride_counters():
    """Section 4's counter increments other than one (stride 3 and 2^20+1)."""
    key = int(oracle.make_keys(4, 1)[0])
    for stride in (3, (1 << 20) + 1):
        ctrs = (np.arange(1 << 18, dtype=np.uint64) * np.uint64(stride))
        out = oracle.pairs32(ctrs, np.uint64(key))
        b = out.view(np.uint8)
        assert abs(pins.chi2_dev(np.bincount(b, minlength=256), b.size)) < 6.0


def test_fill_matches_scalar(rng):
    """The array fill is the scalar generator at consecutive counters,
    wrapping modulo 2^64."""
    key = int(oracle.make_keys(9, 1)[0])
    base = (1 << 64) - 37
    a32 = oracle.fill32(key, base, 100)
    a64 = oracle.fill64(key, base, 100)
    for i in range(100):
        c = (base + i) % (1 << 64)
        assert int(a32[i]) == oracle.squares32(c, key)
        assert int(a64[i]) == oracle.squares64(c, key)
    # threaded fill agrees with the single-threaded one on a longer range
    n = (1 << 18) + 13
    assert np.array_equal(oracle.fill32(key, base, n, threads=1),
                          oracle.fill32(key, base, n, threads=7))


def test_squaring_identity_used_by_kernels(rng):
    """(H*2^32 + L)^2 = L^2 + ((2*L*H) mod 2^32) * 2^32 (mod 2^64): the H^2
    term is a multiple of 2^64. A fact of arithmetic; the kernels rely on it."""
    for _ in range(20000):
        x = int(rng.integers(0, 1 << 64, dtype=np.uint64))
        hi, lo = x >> 32, x & 0xFFFFFFFF
        assert (x * x) % (1 << 64) == (lo * lo + ((2 * lo * hi) % (1 << 32) << 32)) % (1 << 64)
