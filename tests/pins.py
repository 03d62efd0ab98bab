"""The oracle's pins, as functions of the generator under test.

Each pin ties squares32 / squares64 (Section 2 / Section 5) to something
other than the oracle's own code: hand-derived worked examples, identities
that follow from the definitions, closed-form special cases, exhaustive
brute force of a reduced-width analogue and chi-square smoke tests. They take
the functions under test as arguments so that ``test_oracle_mutants.py`` can
run the same battery against copies of the oracle with a planted mistake.
"""
from __future__ import annotations

import os

import numpy as np

M64 = (1 << 64) - 1
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

EDGE_CTRS = [0, 1, 2, (1 << 32) - 1, 1 << 32, (1 << 32) + 1, 1 << 63,
             (1 << 63) - 1, M64 - 1, M64]


def load_hand_worked():
    rows = []
    with open(os.path.join(GOLDEN, "hand_worked.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            fn, ctr, key, val = line.split()
            rows.append((fn, int(ctr), int(key), int(val)))
    return rows


def pin_hand_worked(sq32, sq64):
    """Hand-derived worked examples (tests/golden/hand_worked.txt)."""
    rows = load_hand_worked()
    assert len(rows) >= 8
    for fn, ctr, key, val in rows:
        got = sq32(ctr, key) if fn == "squares32" else sq64(ctr, key)
        assert got == val, (fn, ctr, key, got, val)


def pin_high_half(sq32, sq64, rng, n=2000):
    """Section 5 keeps the fourth-round value t whole and xors a 32-bit
    quantity into it, while squares32 returns the upper half of the same t
    (Section 2). Hence upper32(squares64(c, k)) == squares32(c, k)."""
    ctrs = [int(c) for c in rng.integers(0, 1 << 64, n, dtype=np.uint64)] + EDGE_CTRS
    keys = [int(k) for k in rng.integers(0, 1 << 64, len(ctrs), dtype=np.uint64)]
    for c, k in zip(ctrs, keys):
        assert sq64(c, k) >> 32 == sq32(c, k), (c, k)


def pin_zero_key(sq32, sq64):
    """key = 0 makes y = z = 0, every round maps 0 to 0: output 0."""
    for c in EDGE_CTRS + [12345, 987654321987]:
        assert sq32(c, 0) == 0 and sq64(c, 0) == 0, c


def pin_even_key_period(sq32, sq64, rng):
    """For key = 2^v * m the Weyl terms ctr*key and (ctr+1)*key repeat with
    period 2^(64-v) in ctr (Section 2's Weyl argument), so the outputs do."""
    for v in (1, 7, 31, 40, 63):
        m = int(rng.integers(0, 1 << 62)) * 2 + 1
        key = (m << v) & M64
        for c in [int(x) for x in rng.integers(0, 1 << 64, 20, dtype=np.uint64)]:
            c2 = (c + (1 << (64 - v))) & M64
            assert sq32(c2, key) == sq32(c, key), (v, c)
            assert sq64(c2, key) == sq64(c, key), (v, c)


def pin_odd_key_not_periodic(sq32, sq64, rng):
    """An odd key gives a full-period Weyl sequence: shifting the counter by
    2^63 changes y, and the output changes for almost every counter."""
    key = int(rng.integers(0, 1 << 62)) * 2 + 1
    diff32 = diff64 = 0
    cs = [int(x) for x in rng.integers(0, 1 << 64, 200, dtype=np.uint64)]
    for c in cs:
        c2 = (c + (1 << 63)) & M64
        diff32 += sq32(c2, key) != sq32(c, key)
        diff64 += sq64(c2, key) != sq64(c, key)
    assert diff32 >= 195 and diff64 >= 195


def pin_z_term(sq32, sq64, rng, n=400):
    """The generator adds (ctr+1)*key as well as ctr*key (Section 3). Choose
    (c1, k1), (c2, k2) with odd k1 != k2 and c2*k2 == c1*k1 (mod 2^64): y is
    equal, z = y + key is not, so the outputs must differ (a version that
    only used y would return equal outputs for every such pair)."""
    same = 0
    for _ in range(n):
        k1 = int(rng.integers(0, 1 << 62)) * 2 + 1
        k2 = int(rng.integers(0, 1 << 62)) * 2 + 1
        c1 = int(rng.integers(0, 1 << 64, dtype=np.uint64))
        c2 = (c1 * k1 * pow(k2, -1, 1 << 64)) & M64
        assert (c2 * k2) & M64 == (c1 * k1) & M64
        same += sq32(c1, k1) == sq32(c2, k2)
        same += sq64(c1, k1) == sq64(c2, k2)
    assert same <= 2, same


def _rot_by_multiplication(v: int) -> int:
    """Rotation by 32 bits written as arithmetic: a 64-bit rotation is
    multiplication by 2^32 modulo 2^64 - 1 (all-ones is fixed)."""
    return v if v == M64 else (v << 32) % M64


def bigint_squares(ctr: int, key: int):
    """An arbitrary-precision route: exact integer squares reduced modulo
    2^64 by the % operator, rotations by multiplication mod 2^64 - 1, the
    32-bit "upper half" by floor division."""
    y = (ctr * key) % (1 << 64)
    z = ((ctr + 1) * key) % (1 << 64)
    x = y
    for a in (y, z, y):
        x = _rot_by_multiplication((x * x + a) % (1 << 64))
    t = (x * x + z) % (1 << 64)
    x5 = _rot_by_multiplication(t)
    fifth = (x5 * x5 + y) % (1 << 64)
    return t // (1 << 32), t ^ (fifth // (1 << 32))


def pin_bigint_route(sq32, sq64, rng, n=1500):
    ctrs = [int(c) for c in rng.integers(0, 1 << 64, n, dtype=np.uint64)] + EDGE_CTRS
    keys = [int(k) for k in rng.integers(0, 1 << 64, len(ctrs), dtype=np.uint64)]
    keys[:len(EDGE_CTRS)] = [1, M64, 1 << 32, (1 << 32) + 1, 3, 0x9E3779B97F4A7C15,
                             M64 - 2, 1 << 63, 5, 7][:len(EDGE_CTRS)]
    for c, k in zip(ctrs, keys):
        e32, e64 = bigint_squares(c, k)
        assert sq32(c, k) == e32, (c, k)
        assert sq64(c, k) == e64, (c, k)


def chi2_dev(hist: np.ndarray, total: int) -> float:
    """(chi^2 - dof) / sqrt(2 dof) against the uniform distribution."""
    h = hist.astype(np.float64)
    e = total / h.size
    chi = float(((h - e) ** 2 / e).sum())
    dof = h.size - 1
    return (chi - dof) / np.sqrt(2 * dof)


def reduced_keys(w: int, n: int, rng) -> list[int]:
    """Keys for a w-bit state built like Section 3's: non-zero hex digits,
    distinct within each half, odd last digit."""
    nib = w // 4
    n_low = nib // 2
    n_up = nib - n_low
    keys = []
    while len(keys) < n:
        up = rng.permutation(np.arange(1, 16))[:n_up]
        low = list(rng.permutation(np.arange(1, 16))[: n_low - 1])
        odd = [d for d in range(1, 16, 2) if d not in low]
        low.append(int(rng.choice(odd)))
        digits = list(up) + low
        k = 0
        for d in digits:
            k = (k << 4) | int(d)
        keys.append(k)
    return keys


def pin_reduced_width_uniform(hist_w, rng, w=24, nkeys=6, spread=0.2):
    """Exhaustive brute force of the w-bit analogue over all 2^w counters:
    with odd keys the w/2-bit output is statistically uniform (Section 2
    footnote: each output has probability 2^-(w/2)); with an even key the
    Weyl term loses its full period and uniformity fails (chi^2 > 10 sigma);
    and the per-key histograms differ, as they must when z = y + key
    enters (a y-only generator gives the same histogram for every odd key)."""
    keys = reduced_keys(w, nkeys, rng)
    hists = []
    for k in keys:
        h = hist_w(k, w, 4, True)
        hists.append(h)
        assert abs(chi2_dev(h, 1 << w)) < 6.0, (hex(k), chi2_dev(h, 1 << w))
        e = (1 << w) / h.size
        assert (1 - spread) * e < h.min() and h.max() < (1 + spread) * e
    for i in range(1, len(hists)):
        assert not np.array_equal(hists[0], hists[i])
    even = hist_w(keys[0] ^ 1, w, 4, True)
    assert chi2_dev(even, 1 << w) > 10.0


def pin_reduced_width_is_full_width(squares_w, sq32, sq64, rng, n=300):
    """At w = 64 the analogue is the generator itself (four rounds narrow,
    five rounds wide)."""
    for _ in range(n):
        c = int(rng.integers(0, 1 << 64, dtype=np.uint64))
        k = int(rng.integers(0, 1 << 64, dtype=np.uint64))
        assert squares_w(c, k, 64, 4, True, False) == sq32(c, k)
        assert squares_w(c, k, 64, 5, True, True) == sq64(c, k)


def pin_byte_chi2(fill32, fill64, key: int, base: int, n: int = 1 << 20):
    """Chi-square smoke on output bytes and per-bit frequencies."""
    for arr in (fill32(key, base, n), fill64(key, base, n // 2)):
        b = arr.view(np.uint8)
        assert abs(chi2_dev(np.bincount(b, minlength=256), b.size)) < 6.0
        bits = np.unpackbits(b).reshape(-1, arr.itemsize * 8).mean(axis=0)
        sigma = 0.5 / np.sqrt(arr.size)
        assert np.all(np.abs(bits - 0.5) < 6 * sigma)


def run_scalar_battery(sq32, sq64, seed=20040627):
    """All pins that need only the two scalar functions."""
    rng = np.random.default_rng(seed)
    pin_hand_worked(sq32, sq64)
    pin_high_half(sq32, sq64, rng, n=300)
    pin_zero_key(sq32, sq64)
    pin_even_key_period(sq32, sq64, rng)
    pin_odd_key_not_periodic(sq32, sq64, rng)
    pin_z_term(sq32, sq64, rng, n=100)


# --- Box-Muller on 32-bit halves --------------------------------------------

def pin_box_muller_closed_forms(bm):
    """u1 = 1 gives the origin; lo = 0, 2^30, 2^31, 3*2^30 put the pair on
    the axes; hi = 0 gives the largest radius sqrt(64 ln 2); hi = 2^31 - 1
    gives u1 = 1/2, radius sqrt(2 ln 2); lo = 2^29 is the diagonal."""
    M = (1 << 32) - 1
    hi = np.array([M, M, 0, 0, 0, 0, (1 << 31) - 1, (1 << 31) - 1], dtype=np.uint32)
    lo = np.array([0, 12345, 0, 1 << 30, 1 << 31, 3 << 30, 1 << 29, 0], dtype=np.uint32)
    z = bm(hi, lo)
    rmax, rhalf = np.sqrt(64 * np.log(2)), np.sqrt(2 * np.log(2))
    want = np.array([[0, 0], [0, 0], [rmax, 0], [0, rmax], [-rmax, 0], [0, -rmax],
                     [rhalf / np.sqrt(2), rhalf / np.sqrt(2)], [rhalf, 0]])
    assert np.allclose(z, want, rtol=0, atol=1e-14), z


def pin_box_muller_polar(bm, rng, n=5000):
    """Radius and angle recovered from the pairs of random halves:
    r^2 = -2 ln((hi + 1) / 2^32), angle = 2 pi lo / 2^32."""
    hi = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    lo = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    z = bm(hi, lo)
    r2 = z[:, 0] ** 2 + z[:, 1] ** 2
    assert np.allclose(r2, -2 * np.log((hi.astype(np.float64) + 1) / 2 ** 32), rtol=1e-12, atol=1e-12)
    ang = np.mod(np.arctan2(z[:, 1], z[:, 0]), 2 * np.pi)
    dang = np.angle(np.exp(1j * (ang - 2 * np.pi * lo.astype(np.float64) / 2 ** 32)))
    assert np.all(np.abs(dang[r2 > 1e-6]) < 1e-9)


def run_box_muller_battery(bm, seed=20040627):
    pin_box_muller_closed_forms(bm)
    pin_box_muller_polar(bm, np.random.default_rng(seed))
